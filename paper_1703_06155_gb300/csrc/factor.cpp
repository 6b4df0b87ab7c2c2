// h2_factorize: Algorithm 1 of the paper, run level by level on the GPU.
//
// For each level l = L .. l0 and each elimination batch (a colour class of
// the near-field graph, or a single cluster in the natural order):
//   Phase A (FP64, rank decisions)
//     Step 1 first half: Householder complement Vp of the incoming basis B_i
//     Step 0: M = sum F F^H + sum F^T conj(F) over the live fill-ins of row /
//             column i (eq. 16), G = Vp^H M Vp (eq. 16 in complement
//             coordinates), Jacobi eigen-decomposition (eq. 17), r = number
//             of eigenvalues above eps^2 nu_i^2, Y = Vp U
//   -- host reads r back (one sync per batch) --
//   Phase B (bulk precision)
//     Q~_i = [Y(:, r:), B_i, Y(:, :r)]  (eqs. 18-19: V~ = [V, V_add] kept
//             verbatim as the last k~ columns)
//     Step 2: Q~^H on block row i, conj(Q~) on block column i (eq. 5, Alg. 3)
//     Step 3: LU of the leading m x m block with L^{-1}P, U^{-1} (eq. 11),
//             panels L^{-1}P Z_i'c and Z_ci' U^{-1} (Alg. 4 l.2-3), Schur
//             updates grouped by target block (Alg. 4 l.4, eqs. 12, 15)
// After the level: couplings pad(S) + F (eqs. 20-22, 33) and padded transfers
// (eq. 23) are written straight into the merged parent blocks (Fig. 2 g-i).
// After level l0: blocked LU of the final block.
//
// Blocks live in place: at the end of a level the near-field arena holds the
// U panels (rows 0..m_i of block row i), the L panels (columns 0..m_i of
// block column i) and the LU of each diagonal block, i.e. the factors L_i^l,
// U_i^l of eq. 34; Q~_i, L^{-1}P, U^{-1} and the pivots sit in their own
// arenas.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <set>

#include "batch.h"

namespace h2 {
using namespace h2k;

void run_gemm(Ctx& c, GemmBatch& b, int pin, int pout, int pacc, const char* what) {
  if (b.empty()) return;
  const int64_t ws = b.plan();
  if (b.tl.empty()) return;
  void* wsp = nullptr;
  if (ws > 0) wsp = dev_ensure(c, c.gemm_ws, (size_t)ws * (pacc == P64 ? sizeof(cd) : sizeof(cf)));
  const int i0 = c.st.add(b.t), i1 = c.st.add(b.p), i2 = c.st.add(b.tl);
  c.st.upload(c);
  ProfScope ps(c, std::string("gemm:") + what, b.alg_flops);
  ck(gemm(c.st.ptr<GemmTask>(i0), c.st.ptr<GemmPair>(i1), c.st.ptr<GemmTile>(i2), (int)b.tl.size(), pin, pout, pacc,
          wsp, c.stream, b.skinny),
     what);
  c.launches++;
  if (ws > 0) {
    int maxmn = 0;
    for (auto& g : b.t)
      if (g.nk > 1) maxmn = std::max(maxmn, g.M * g.N);
    ck(gemm_reduce(c.st.ptr<GemmTask>(i0), (int)b.t.size(), maxmn, pout, pacc, wsp, c.stream), what);
    c.launches++;
  }
  int maxh = 0;
  for (auto& g : b.t)
    if (g.herm) maxh = std::max(maxh, g.M * g.N);
  if (maxh > 0) {
    ck(gemm_mirror(c.st.ptr<GemmTask>(i0), (int)b.t.size(), maxh, pout, c.stream), what);
    c.launches++;
  }
}

void run_apply(Ctx& c, ApplyBatch& b, bool left, int prec, const char* what) {
  if (b.empty()) return;
  const int tw = apply_tile_width(prec, b.maxp);
  std::vector<ApplyTile> tiles;
  for (size_t i = 0; i < b.t.size(); ++i)
    for (int t0 = 0; t0 < b.t[i].w; t0 += tw) tiles.push_back(ApplyTile{(int)i, t0});
  const int i0 = c.st.add(b.t), i1 = c.st.add(tiles);
  c.st.upload(c);
  ProfScope ps(c, std::string(left ? "apply_left:" : "apply_right:") + what, b.flops);
  if (left)
    ck(apply_left(c.st.ptr<ApplyTask>(i0), c.st.ptr<ApplyTile>(i1), (int)tiles.size(), prec, b.maxp, tw, c.stream),
       what);
  else
    ck(apply_right(c.st.ptr<ApplyTask>(i0), c.st.ptr<ApplyTile>(i1), (int)tiles.size(), prec, b.maxp, tw, c.stream),
       what);
  c.launches++;
}

void run_apply_gemm(Ctx& c, ApplyBatch& b, bool left, int prec, const char* what) {
  if (b.empty()) return;
  const size_t es = esz(prec);
  std::vector<size_t> off;
  size_t tot = 0;
  for (const ApplyTask& t : b.t) {
    off.push_back(tot);
    tot += ((size_t)(t.p - t.lo) * t.w + 31) / 32 * 32;
  }
  char* W = (char*)dev_ensure(c, c.applybuf, tot * es);
  GemmBatch g;
  CopyBatch cb;
  for (size_t i = 0; i < b.t.size(); ++i) {
    const ApplyTask& t = b.t[i];
    const int out = t.p - t.lo;
    const bool tr = t.opA == OP_T || t.opA == OP_H;
    if (left) {
      // W (out x w) = op(A)[lo:p, 0:p] X[0:p, :]
      const char* A = (const char*)t.A + (tr ? (size_t)t.lo * t.lda : (size_t)t.lo) * es;
      g.task(W + off[i] * es, out, out, t.w, 1.0, 0.0);
      g.pair(A, t.lda, t.opA, t.X, t.ldx, OP_N, t.p);
      g.close();
      cb.add(W + off[i] * es, prec, out, out, t.w, (char*)t.X + (size_t)t.lo * es, prec, t.ldx, out, t.w);
    } else {
      // W (w x out) = X[:, 0:p] op(A)[0:p, lo:p]
      const char* A = (const char*)t.A + (tr ? (size_t)t.lo : (size_t)t.lo * t.lda) * es;
      g.task(W + off[i] * es, t.w, t.w, out, 1.0, 0.0);
      g.pair(t.X, t.ldx, OP_N, A, t.lda, t.opA, t.p);
      g.close();
      cb.add(W + off[i] * es, prec, t.w, t.w, out, (char*)t.X + (size_t)t.lo * t.ldx * es, prec, t.ldx, t.w, out);
    }
  }
  run_gemm(c, g, prec, prec, prec, what);
  run_copy(c, cb, what);
}

void run_copy(Ctx& c, CopyBatch& b, const char* what) {
  if (b.empty()) return;
  const int i0 = c.st.add(b.t);
  c.st.upload(c);
  ProfScope ps(c, std::string("copy:") + what, 0.0);
  ck(copy2d(c.st.ptr<CopyTask>(i0), (int)b.t.size(), c.stream), what);
  c.launches++;
}

namespace {

// Step 2 / panel applications: in-place kernel or GEMM + copy (h2_opts.apply_path)
void run_apply_auto(Ctx& c, ApplyBatch& b, bool left, int prec, const char* what) {
  if (c.opts.apply_path == 1) run_apply(c, b, left, prec, what);
  else run_apply_gemm(c, b, left, prec, what);
}

void setup_level(Ctx& c, LevelF& F, int l, const std::vector<int>& n, const std::vector<Pair>& carried) {
  const H2Host& H = c.H;
  const int nc = 1 << l;
  {
    // keep the device arenas of an earlier factorization (grow-only)
    DevBuf b1 = std::move(F.near_buf), b2 = std::move(F.fill_buf), b3 = std::move(F.B_buf), b4 = std::move(F.Q_buf),
           b5 = std::move(F.inv_buf), b6 = std::move(F.piv_buf), b7 = std::move(F.Ub_buf), b8 = std::move(F.Vp_buf);
    F = LevelF();
    F.near_buf = std::move(b1);
    F.fill_buf = std::move(b2);
    F.B_buf = std::move(b3);
    F.Q_buf = std::move(b4);
    F.inv_buf = std::move(b5);
    F.piv_buf = std::move(b6);
    F.Ub_buf = std::move(b7);
    F.Vp_buf = std::move(b8);
  }
  F.l = l;
  F.nc = nc;
  F.n = n;
  F.k0 = H.rank[l];
  F.kt = F.k0;
  F.m.assign(nc, 0);
  F.nbrs = near_lists(H.part, l);
  if (c.opts.ordering == H2_ORDER_NATURAL) {
    for (int i = 0; i < nc; ++i) F.batches.push_back({i});
  } else {
    const std::vector<int> col = greedy_colours(F.nbrs);
    const int ncol = *std::max_element(col.begin(), col.end()) + 1;
    F.batches.assign(ncol, {});
    for (int i = 0; i < nc; ++i) F.batches[col[i]].push_back(i);
  }
  F.nbr_first.assign(nc + 1, 0);
  for (int i = 0; i < nc; ++i) F.nbr_first[i + 1] = F.nbr_first[i] + (int)F.nbrs[i].size();
  F.batch_of.assign(nc, 0);
  for (size_t b = 0; b < F.batches.size(); ++b)
    for (int i : F.batches[b]) F.batch_of[i] = (int)b;
  const size_t es = esz(c.prec);
  // near-field blocks (inadmissible at this level)
  F.near_pairs = H.part.inad[l];
  size_t tot = 0;
  for (size_t q = 0; q < F.near_pairs.size(); ++q) {
    const auto [a, b] = F.near_pairs[q];
    F.near_id[pkey(a, b)] = (int)q;
    F.near_off.push_back(tot);
    tot += (size_t)n[a] * n[b];
  }
  dev_ensure(c, F.near_buf, tot * es);
  // fill-in blocks: every Schur target outside the near field, plus the
  // fill-ins carried up from the children of pushed blocks
  std::set<Pair> fs(carried.begin(), carried.end());
  for (int i = 0; i < nc; ++i)
    for (int j : F.nbrs[i])
      for (int k : F.nbrs[i])
        if (!F.near_id.count(pkey(j, k))) fs.insert({j, k});
  F.fill_pairs.assign(fs.begin(), fs.end());
  std::set<Pair> cs(carried.begin(), carried.end());
  tot = 0;
  for (size_t q = 0; q < F.fill_pairs.size(); ++q) {
    const auto [a, b] = F.fill_pairs[q];
    F.fill_id[pkey(a, b)] = (int)q;
    F.fill_off.push_back(tot);
    F.fill_live.push_back(cs.count(F.fill_pairs[q]) ? 1 : 0);
    F.fill_is_adm.push_back(c.adm_id[l].count(pkey(a, b)) ? 1 : 0);
    tot += (size_t)n[a] * n[b];
  }
  dev_ensure(c, F.fill_buf, tot * es);
  if (tot) ck(cudaMemsetAsync(F.fill_buf.p, 0, tot * es, c.stream), "fill memset");
  // bases (FP64), Q (bulk), L^{-1}P and U^{-1} (bulk), pivots
  size_t tb = 0, tq = 0, ti = 0, tp = 0, tvp = 0;
  F.voff.assign(nc, 0);
  F.vlen = 0;
  for (int i = 0; i < nc; ++i) {
    if (F.k0[i] > 1024 || n[i] > 4096)
      fail(H2_EINTERNAL, "cluster size " + std::to_string(n[i]) + " / rank " + std::to_string(F.k0[i]) +
                             " above the kernel limits (4096 / 1024)");
    F.B_off.push_back(tb);
    tb += (size_t)n[i] * F.k0[i];
    F.Q_off.push_back(tq);
    tq += (size_t)n[i] * n[i];
    F.inv_off.push_back(ti);
    ti += 2 * (size_t)n[i] * n[i];
    F.piv_off.push_back(tp);
    tp += n[i];
    F.Vp_off.push_back(tvp);
    tvp += (size_t)n[i] * (n[i] - F.k0[i]);
    F.voff[i] = F.vlen;
    F.vlen += n[i];
  }
  dev_ensure(c, F.B_buf, tb * sizeof(cd));
  dev_ensure(c, F.Q_buf, tq * es);
  dev_ensure(c, F.inv_buf, ti * es);
  dev_ensure(c, F.piv_buf, tp * sizeof(int));
  dev_ensure(c, F.Vp_buf, tvp * sizeof(cd));
  // sum of ||S||_F^2 over the admissible blocks of each row and column
  F.snorm2.assign(nc, 0.0);
  for (size_t q = 0; q < H.part.adm[l].size(); ++q) {
    double v = 0;
    for (const cplx& z : H.S[l][q]) v += std::norm(z);
    F.snorm2[H.part.adm[l][q].first] += v;
    F.snorm2[H.part.adm[l][q].second] += v;
  }
}

struct Ptrs {
  char* near;
  char* fill;
  cd* B;
  char* Q;
  char* inv;
  int* piv;
  size_t es;
};

Ptrs ptrs(Ctx& c, LevelF& F) {
  return Ptrs{(char*)F.near_buf.p, (char*)F.fill_buf.p, (cd*)F.B_buf.p, (char*)F.Q_buf.p, (char*)F.inv_buf.p,
              (int*)F.piv_buf.p, esz(c.prec)};
}

void process_batch(Ctx& c, LevelF& F, const std::vector<int>& bt, std::vector<char>& done, double eps) {
  const int prec = c.prec;
  Ptrs P = ptrs(c, F);
  const size_t es = P.es;
  auto NB = [&](int j, int k) -> char* { return P.near + F.near_off.at(F.near_id.at(pkey(j, k))) * es; };
  auto FB = [&](int id) -> char* { return P.fill + F.fill_off[id] * es; };
  auto lo_of = [&](int j) { return done[j] ? F.m[j] : 0; };
  std::set<int> inb(bt.begin(), bt.end());

  // ------------------------------ Phase A (FP64) ---------------------------
  // Vp: complement of the incoming basis (stored with the level); G' = Vp^H M
  // Vp is the Gram of eq. (16) in complement coordinates.
  struct Info {
    int i, n, k0, p, rp = 0;
    bool fill;
    size_t M, T1, G, L, T, W, Qx, Z1, Gh, U, lam, W1, W2, Yf, Y1;
    std::vector<int> rowf, colf;
  };
  std::vector<Info> info;
  size_t sc = 0;  // scratch in cd units
  for (int i : bt) {
    Info f{};
    f.i = i;
    f.n = F.n[i];
    f.k0 = F.k0[i];
    f.p = f.n - f.k0;
    for (size_t q = 0; q < F.fill_pairs.size(); ++q) {
      if (!F.fill_live[q]) continue;
      if (F.fill_pairs[q].first == i) f.rowf.push_back((int)q);
      if (F.fill_pairs[q].second == i) f.colf.push_back((int)q);
    }
    f.fill = (!f.rowf.empty() || !f.colf.empty()) && f.p > 0;
    if (f.fill) {
      const size_t n = f.n, p = f.p;
      auto take = [&](size_t cnt) { const size_t o = sc; sc += cnt; return o; };
      f.M = take(n * n);
      f.T1 = take(n * p);
      f.G = take(p * p);
      f.L = take(p * p);
      f.T = take(p * p);
      f.W = take(p * p);
      f.Qx = take(p * p);
      f.Z1 = take(p * p);
      f.Gh = take(p * p);
      f.U = take(p * p);
      f.lam = take(p / 2 + 1);
      f.W1 = take(n * p);
      f.W2 = take(n * p);
      f.Yf = take(n * p);
      f.Y1 = take(n * p);
    }
    info.push_back(f);
  }
  cd* S = (cd*)dev_ensure(c, c.scratch, (sc + 1) * sizeof(cd));
  int* d_r = (int*)dev_ensure(c, c.normbuf, 3 * bt.size() * sizeof(int) + 64);
  ck(cudaMemsetAsync(d_r, 0, 3 * bt.size() * sizeof(int), c.stream), "memset r");
  auto Vp = [&](int i) { return (cd*)F.Vp_buf.p + F.Vp_off[i]; };
  // With a symmetric Z the column fill-ins are the transposed row fill-ins and
  // the column Gram equals the row Gram: only the row side is formed, and the
  // admissible-row norm is halved to match (the decisions are unchanged).
  auto snorm = [&](int i) { return c.H.symmetric ? 0.5 * F.snorm2[i] : F.snorm2[i]; };
  bool anyfill = false;
  for (auto& f : info) anyfill |= f.fill;
  std::vector<int> r(bt.size(), 0), sweeps;
  if (anyfill) {
    GemmBatch gM, gT, gG;
    std::vector<PcholTask> pc;
    int maxp = 0;
    for (size_t q = 0; q < info.size(); ++q) {
      Info& f = info[q];
      if (!f.fill) continue;
      const int n = f.n;
      gM.task(S + f.M, n, n, n, 1.0, 0.0);
      for (int id : f.rowf) {
        const int k = F.fill_pairs[id].second, lo = lo_of(k);
        char* A = FB(id) + (size_t)lo * n * es;
        gM.pair(A, n, OP_N, A, n, OP_H, F.n[k] - lo);
      }
      if (!c.H.symmetric)
        for (int id : f.colf) {
          const int k = F.fill_pairs[id].first, lo = lo_of(k);
          char* A = FB(id) + (size_t)lo * es;
          gM.pair(A, F.n[k], OP_T, A, F.n[k], OP_C, F.n[k] - lo);
        }
      gM.hermitian();
      gM.close();
      gT.task(S + f.T1, n, n, f.p, 1.0, 0.0);
      gT.pair(S + f.M, n, OP_N, Vp(f.i), n, OP_N, n);
      gT.close();
      gG.task(S + f.G, f.p, f.p, f.p, 1.0, 0.0);
      gG.pair(Vp(f.i), n, OP_H, S + f.T1, n, OP_N, n);
      gG.close();
      pc.push_back(PcholTask{S + f.G, S + f.M, S + f.L, S + f.T, d_r + q, f.p, n, snorm(f.i), eps * eps});
      maxp = std::max(maxp, f.p);
    }
    run_gemm(c, gM, prec, P64, P64, "gram");
    run_gemm(c, gT, P64, P64, P64, "gram*Vp");
    run_gemm(c, gG, P64, P64, P64, "Vp^H*gram*Vp");
    {
      const int i0 = c.st.add(pc);
      c.st.upload(c);
      ProfScope ps(c, "pchol_wy", 0.0);
      ck(pchol_wy(c.st.ptr<PcholTask>(i0), (int)pc.size(), maxp, c.stream), "pivoted cholesky");
      c.launches++;
    }
    std::vector<int> rp(bt.size(), 0);
    ck(cudaMemcpyAsync(rp.data(), d_r, bt.size() * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "read r'");
    ck(cudaStreamSynchronize(c.stream), "sync after pivoted cholesky");
    c.st.begin();
    for (size_t q = 0; q < info.size(); ++q)
      if (info[q].fill) info[q].rp = std::min(std::max(rp[q], 0), info[q].p);
    // Ritz step on span(Qx) and the complement rotation Yf = Vp Q, Q = I - Y T Y^H
    GemmBatch g1, g2, g3, g4, g5;
    CopyBatch cp;
    std::vector<EigTask> eig;
    std::vector<SelTask> sel;
    int maxr = 0;
    for (size_t q = 0; q < info.size(); ++q) {
      Info& f = info[q];
      if (!f.fill || f.rp == 0) continue;
      const int n = f.n, p = f.p, rr = f.rp;
      cd* Y = S + f.L;
      g1.task(S + f.W, p, p, rr, 1.0, 0.0);  // W = Y T
      g1.pair(Y, p, OP_N, S + f.T, rr, OP_N, rr);
      g1.close();
      g1.task(S + f.W1, n, n, rr, 1.0, 0.0);  // W1 = Vp Y
      g1.pair(Vp(f.i), n, OP_N, Y, p, OP_N, p);
      g1.close();
      cp.add(nullptr, P64, p, 0, 0, S + f.Qx, P64, p, p, rr, 2);                  // Qx = E
      cp.add(Vp(f.i), P64, n, n, p, S + f.Yf, P64, n, n, p, 0);                   // Yf = Vp
      g2.task(S + f.Qx, p, p, rr, -1.0, 1.0);  // Qx = E - W Y(0:r',:)^H
      g2.pair(S + f.W, p, OP_N, Y, p, OP_H, rr);
      g2.close();
      g2.task(S + f.W2, n, n, rr, 1.0, 0.0);  // W2 = W1 T
      g2.pair(S + f.W1, n, OP_N, S + f.T, rr, OP_N, rr);
      g2.close();
      g3.task(S + f.Z1, p, p, rr, 1.0, 0.0);  // Z1 = G' Qx
      g3.pair(S + f.G, p, OP_N, S + f.Qx, p, OP_N, p);
      g3.close();
      g3.task(S + f.Yf, n, n, p, -1.0, 1.0);  // Yf = Vp - W2 Y^H
      g3.pair(S + f.W2, n, OP_N, Y, p, OP_H, rr);
      g3.close();
      g4.task(S + f.Gh, rr, rr, rr, 1.0, 0.0);  // Ritz matrix Qx^H G' Qx
      g4.pair(S + f.Qx, p, OP_H, S + f.Z1, p, OP_N, p);
      g4.close();
      eig.push_back(EigTask{S + f.Gh, S + f.U, (double*)(S + f.lam), rr, d_r + 2 * bt.size() + q});
      sel.push_back(SelTask{S + f.M, (double*)(S + f.lam), d_r + bt.size() + q, n, rr, snorm(f.i), eps * eps});
      maxr = std::max(maxr, rr);
      g5.task(S + f.Y1, n, n, rr, 1.0, 0.0);  // Y1 = Yf(:, 0:r') U
      g5.pair(S + f.Yf, n, OP_N, S + f.U, rr, OP_N, rr);
      g5.close();
    }
    run_gemm(c, g1, P64, P64, P64, "WY 1");
    run_copy(c, cp, "WY presets");
    run_gemm(c, g2, P64, P64, P64, "WY 2");
    run_gemm(c, g3, P64, P64, P64, "WY 3");
    run_gemm(c, g4, P64, P64, P64, "ritz matrix");
    if (!eig.empty()) {
      const int i0 = c.st.add(eig);
      c.st.upload(c);
      ProfScope ps(c, maxr >= 48 ? "jacobi_cluster" : "jacobi", 0.0);
      if (maxr >= 48) {
        // large Ritz problems: one 8-CTA cluster per eigenproblem
        const int64_t per = jacobi_cluster_scratch(maxr);
        double* js = (double*)dev_ensure(c, c.jac_buf, (size_t)per * eig.size() * sizeof(double));
        ck(jacobi_eig_cluster(c.st.ptr<EigTask>(i0), (int)eig.size(), maxr, 8, js, (int*)c.statusbuf.p, c.stream),
           "jacobi (cluster)");
      } else {
        ck(jacobi_eig(c.st.ptr<EigTask>(i0), (int)eig.size(), maxr, (int*)c.statusbuf.p, c.stream), "jacobi");
      }
      c.launches++;
      const int i1 = c.st.add(sel);
      c.st.upload(c);
      ck(select_rank(c.st.ptr<SelTask>(i1), (int)sel.size(), c.stream), "select");
      c.launches++;
    }
    run_gemm(c, g5, P64, P64, P64, "ritz vectors");
    ck(cudaMemcpyAsync(r.data(), d_r + bt.size(), bt.size() * sizeof(int), cudaMemcpyDeviceToHost, c.stream),
       "read r");
    sweeps.resize(bt.size());
    ck(cudaMemcpyAsync(sweeps.data(), d_r + 2 * bt.size(), bt.size() * sizeof(int), cudaMemcpyDeviceToHost, c.stream),
       "read sweeps");
  }
  ck(cudaStreamSynchronize(c.stream), "sync after step 0");
  prof_resolve(c);
  c.st.begin();  // stream idle: staging can be reused
  for (size_t q = 0; q < info.size(); ++q) {
    const Info& f = info[q];
    const int rr = (f.fill && f.rp > 0) ? std::min(std::max(r[q], 0), f.rp) : 0;
    if (f.fill && f.rp > 0) {
      F.st_ritz_max = std::max(F.st_ritz_max, f.rp);
      F.st_ritz_sum += f.rp;
      F.st_ritz_n++;
      if (!sweeps.empty()) F.st_sweeps_max = std::max(F.st_sweeps_max, sweeps[q]);
    }
    r[q] = rr;
    F.kt[f.i] = f.k0 + rr;
    F.m[f.i] = f.n - F.kt[f.i];
  }

  // ------------------------------ Phase B (bulk) ---------------------------
  CopyBatch qc;
  for (size_t q = 0; q < info.size(); ++q) {
    const Info& f = info[q];
    const int n = f.n, m = F.m[f.i], rr = r[q];
    char* Q = P.Q + F.Q_off[f.i] * es;
    if (f.fill && f.rp > 0) {
      // Q~ = [Y1(:, r:r'), Yf(:, r':p), B, Y1(:, 0:r)]  (eqs. 18-19)
      const int rp = f.rp;
      qc.add(S + f.Y1 + (size_t)rr * n, P64, n, n, rp - rr, Q, prec, n, n, rp - rr);
      qc.add(S + f.Yf + (size_t)rp * n, P64, n, n, f.p - rp, Q + (size_t)(rp - rr) * n * es, prec, n, n, f.p - rp);
      if (rr > 0) qc.add(S + f.Y1, P64, n, n, rr, Q + (size_t)(m + f.k0) * n * es, prec, n, n, rr);
    } else {
      qc.add(Vp(f.i), P64, n, n, f.p, Q, prec, n, n, f.p);
    }
    qc.add(P.B + F.B_off[f.i], P64, n, n, f.k0, Q + (size_t)m * n * es, prec, n, n, f.k0);
  }
  run_copy(c, qc, "form Q");

  // Step 2: rows (left, Q^H) then columns (right, conj Q)
  ApplyBatch L2, R2;
  for (int i : bt) {
    const int n = F.n[i], m = F.m[i];
    const char* Q = P.Q + F.Q_off[i] * es;
    for (int j : F.nbrs[i]) {
      if (j == i) {
        L2.add(Q, n, OP_H, NB(i, i), n, n, n, 0);
        R2.add(Q, n, OP_C, NB(i, i), n, n, n, 0);
      } else {
        const int lo = lo_of(j);
        L2.add(Q, n, OP_H, NB(i, j) + (size_t)lo * n * es, n, n, F.n[j] - lo, 0);
        R2.add(Q, n, OP_C, NB(j, i) + (size_t)lo * es, F.n[j], n, F.n[j] - lo, 0);
      }
    }
    for (size_t id = 0; id < F.fill_pairs.size(); ++id) {
      if (!F.fill_live[id]) continue;
      const auto [a, b] = F.fill_pairs[id];
      if (a == i) {
        const int lo = lo_of(b);
        L2.add(Q, n, OP_H, FB((int)id) + (size_t)lo * n * es, n, n, F.n[b] - lo, m);
      }
      if (b == i) {
        const int lo = lo_of(a);
        R2.add(Q, n, OP_C, FB((int)id) + (size_t)lo * es, F.n[a], n, F.n[a] - lo, m);
      }
    }
  }
  run_apply_auto(c, L2, true, prec, "step2 rows");
  run_apply_auto(c, R2, false, prec, "step2 cols");
  c.stats.flops_factor += L2.flops + R2.flops;

  // Step 3: LU + explicit inverses, panels, Schur
  std::vector<LuTask> lu;
  for (int i : bt) {
    const int n = F.n[i], m = F.m[i];
    if (m <= 0) continue;
    char* inv = P.inv + F.inv_off[i] * es;
    lu.push_back(LuTask{NB(i, i), inv, inv + (size_t)n * n * es, P.piv + F.piv_off[i], n, m});
    c.stats.flops_factor += 8.0 / 3.0 * m * (double)m * m + 8.0 / 3.0 * m * (double)m * m;
  }
  if (!lu.empty()) {
    const int i0 = c.st.add(lu);
    c.st.upload(c);
    ProfScope ps(c, "lu", 0.0);
    int maxm = 0;
    for (const LuTask& q : lu) maxm = std::max(maxm, q.m);
    ck(lu_blocked(c.st.ptr<LuTask>(i0), (int)lu.size(), maxm, prec, (int*)c.statusbuf.p, c.stream), "lu");
    c.launches++;
  }
  ApplyBatch PL, PR;
  for (int i : bt) {
    const int n = F.n[i], m = F.m[i];
    if (m <= 0) continue;
    const char* Linv = P.inv + F.inv_off[i] * es;
    const char* Uinv = Linv + (size_t)n * n * es;
    for (int j : F.nbrs[i]) {
      const int lo = (j == i) ? m : lo_of(j);
      PL.add(Linv, m, OP_N, NB(i, j) + (size_t)lo * n * es, n, m, F.n[j] - lo, 0);
      PR.add(Uinv, m, OP_N, NB(j, i) + (size_t)lo * es, F.n[j], m, F.n[j] - lo, 0);
    }
  }
  run_apply_auto(c, PL, true, prec, "U panels");
  run_apply_auto(c, PR, false, prec, "L panels");
  c.stats.flops_factor += PL.flops + PR.flops;

  std::map<int64_t, std::vector<int>> tg;
  for (int i : bt) {
    if (F.m[i] <= 0) continue;
    for (int j : F.nbrs[i])
      for (int k : F.nbrs[i]) tg[pkey(j, k)].push_back(i);
  }
  GemmBatch gs;
  for (auto& [key, cl] : tg) {
    const int j = (int)(key >> 32), k = (int)(uint32_t)key;
    const int rlo = inb.count(j) ? F.m[j] : lo_of(j);
    const int clo = inb.count(k) ? F.m[k] : lo_of(k);
    const int nj = F.n[j], nk = F.n[k];
    char* C;
    auto it = F.near_id.find(key);
    if (it != F.near_id.end()) {
      C = P.near + F.near_off[it->second] * es;
    } else {
      const int id = F.fill_id.at(key);
      C = FB(id);
      F.fill_live[id] = 1;
    }
    gs.task(C + ((size_t)rlo + (size_t)clo * nj) * es, nj, nj - rlo, nk - clo, -1.0, 1.0);
    for (int i : cl) {
      const int ni = F.n[i], mi = F.m[i];
      gs.pair(NB(j, i) + (size_t)rlo * es, nj, OP_N, NB(i, k) + (size_t)clo * ni * es, ni, OP_N, mi);
    }
    gs.close();
  }
  run_gemm(c, gs, prec, prec, prec, "schur");
  c.stats.flops_factor += gs.flops;
  for (int i : bt) done[i] = 1;
}

std::vector<Pair> merge_level(Ctx& c, LevelF& F, LevelF& Pn) {
  const int l = F.l;
  const size_t es = esz(c.prec);
  const int prec = c.prec;
  // parents of live pushed fill-ins carry them into level l-1
  std::set<Pair> carried;
  for (size_t q = 0; q < F.fill_pairs.size(); ++q)
    if (F.fill_live[q] && !F.fill_is_adm[q]) carried.insert({F.fill_pairs[q].first / 2, F.fill_pairs[q].second / 2});
  std::vector<int> n(F.nc / 2);
  for (int p = 0; p < F.nc / 2; ++p) n[p] = F.kt[2 * p] + F.kt[2 * p + 1];
  setup_level(c, Pn, l - 1, n, std::vector<Pair>(carried.begin(), carried.end()));
  Ptrs S = ptrs(c, F), D = ptrs(c, Pn);
  auto NBs = [&](int a, int b) { return S.near + F.near_off.at(F.near_id.at(pkey(a, b))) * es; };
  auto ro = [&](int a) { return (a & 1) ? F.kt[a - 1] : 0; };
  CopyBatch as, ac;
  for (size_t q = 0; q < Pn.near_pairs.size(); ++q) {
    const auto [p, r] = Pn.near_pairs[q];
    char* dst = D.near + Pn.near_off[q] * es;
    const int ld = Pn.n[p];
    for (int a = 2 * p; a <= 2 * p + 1; ++a)
      for (int b = 2 * r; b <= 2 * r + 1; ++b) {
        char* d = dst + ((size_t)ro(a) + (size_t)ro(b) * ld) * es;
        const int64_t key = pkey(a, b);
        if (F.near_id.count(key)) {
          as.add(NBs(a, b) + ((size_t)F.m[a] + (size_t)F.m[b] * F.n[a]) * es, prec, F.n[a], F.kt[a], F.kt[b], d, prec,
                 ld, F.kt[a], F.kt[b]);
        } else {
          const int idx = c.adm_id[l].at(key);
          as.add((char*)c.dS.p + c.S_off[l][idx] * sizeof(cd), P64, F.k0[a], F.k0[a], F.k0[b], d, prec, ld, F.kt[a],
                 F.kt[b]);
          auto it = F.fill_id.find(key);
          if (it != F.fill_id.end() && F.fill_live[it->second])
            ac.add(S.fill + (F.fill_off[it->second] + (size_t)F.m[a] + (size_t)F.m[b] * F.n[a]) * es, prec, F.n[a],
                   F.kt[a], F.kt[b], d, prec, ld, F.kt[a], F.kt[b], 1);
        }
      }
  }
  for (size_t q = 0; q < F.fill_pairs.size(); ++q) {
    if (!F.fill_live[q] || F.fill_is_adm[q]) continue;
    const auto [a, b] = F.fill_pairs[q];
    const int id = Pn.fill_id.at(pkey(a / 2, b / 2));
    const int ld = Pn.n[a / 2];
    char* d = D.fill + (Pn.fill_off[id] + (size_t)ro(a) + (size_t)ro(b) * ld) * es;
    ac.add(S.fill + (F.fill_off[q] + (size_t)F.m[a] + (size_t)F.m[b] * F.n[a]) * es, prec, F.n[a], F.kt[a], F.kt[b],
           d, prec, ld, F.kt[a], F.kt[b], 1);
  }
  // complement of the padded transfer: the stored complement of T (rows of
  // child 1 and child 2 at their places) plus one unit column per padded row
  for (int p = 0; p < Pn.nc; ++p) {
    const int c1 = 2 * p, c2 = 2 * p + 1, kp = Pn.k0[p], np_ = Pn.n[p], pp = np_ - kp;
    if (pp <= 0) continue;
    cd* V = (cd*)Pn.Vp_buf.p + Pn.Vp_off[p];
    as.add(nullptr, P64, np_, 0, 0, V, P64, np_, np_, pp);
    const int q = F.k0[c1] + F.k0[c2] - kp, pad1 = F.kt[c1] - F.k0[c1], pad2 = F.kt[c2] - F.k0[c2];
    const cd* Tp = (const cd*)c.dTp.p + c.Tp_off[l - 1][p];
    const int ldT = F.k0[c1] + F.k0[c2];
    if (q > 0) {
      ac.add(Tp, P64, ldT, F.k0[c1], q, V, P64, np_, F.k0[c1], q, 0);
      ac.add(Tp + F.k0[c1], P64, ldT, F.k0[c2], q, V + F.kt[c1], P64, np_, F.k0[c2], q, 0);
    }
    if (pad1 > 0) ac.add(nullptr, P64, 0, 0, 0, V + F.k0[c1] + (size_t)q * np_, P64, np_, pad1, pad1, 2);
    if (pad2 > 0)
      ac.add(nullptr, P64, 0, 0, 0, V + F.kt[c1] + F.k0[c2] + (size_t)(q + pad1) * np_, P64, np_, pad2, pad2, 2);
  }
  // padded transfers (eq. 23): rows of child 1, then rows of child 2
  for (int p = 0; p < Pn.nc; ++p) {
    const int c1 = 2 * p, c2 = 2 * p + 1, kp = Pn.k0[p];
    if (kp == 0) continue;
    const cd* T = (const cd*)c.dT.p + c.T_off[l - 1][p];
    const int ldT = F.k0[c1] + F.k0[c2];
    cd* Bp = D.B + Pn.B_off[p];
    as.add(T, P64, ldT, F.k0[c1], kp, Bp, P64, Pn.n[p], F.kt[c1], kp);
    as.add(T + F.k0[c1], P64, ldT, F.k0[c2], kp, Bp + F.kt[c1], P64, Pn.n[p], F.kt[c2], kp);
  }
  run_copy(c, as, "merge");
  run_copy(c, ac, "merge fill");
  return {};
}

void root_factor(Ctx& c, LevelF& F) {
  const int prec = c.prec;
  const size_t es = esz(prec);
  const int l = F.l;
  RootF& R = c.root;
  R.kt = F.kt;
  std::vector<int> off(F.nc + 1, 0);
  for (int a = 0; a < F.nc; ++a) off[a + 1] = off[a] + F.kt[a];
  const int n = off[F.nc];
  R.n = n;
  if (n == 0) return;
  char* Rm = (char*)dev_ensure(c, R.R, (size_t)n * n * es);
  Ptrs S = ptrs(c, F);
  CopyBatch as, ac;
  for (int a = 0; a < F.nc; ++a)
    for (int b = 0; b < F.nc; ++b) {
      char* d = Rm + ((size_t)off[a] + (size_t)off[b] * n) * es;
      const int64_t key = pkey(a, b);
      if (F.near_id.count(key)) {
        as.add(S.near + (F.near_off[F.near_id.at(key)] + (size_t)F.m[a] + (size_t)F.m[b] * F.n[a]) * es, prec, F.n[a],
               F.kt[a], F.kt[b], d, prec, n, F.kt[a], F.kt[b]);
      } else {
        auto ai = c.adm_id[l].find(key);
        if (ai == c.adm_id[l].end()) fail(H2_EINTERNAL, "final block: pair neither near nor admissible");
        as.add((char*)c.dS.p + c.S_off[l][ai->second] * sizeof(cd), P64, F.k0[a], F.k0[a], F.k0[b], d, prec, n,
               F.kt[a], F.kt[b]);
        auto it = F.fill_id.find(key);
        if (it != F.fill_id.end() && F.fill_live[it->second])
          ac.add(S.fill + (F.fill_off[it->second] + (size_t)F.m[a] + (size_t)F.m[b] * F.n[a]) * es, prec, F.n[a],
                 F.kt[a], F.kt[b], d, prec, n, F.kt[a], F.kt[b], 1);
      }
    }
  run_copy(c, as, "root assemble");
  run_copy(c, ac, "root assemble fill");
  // blocked right-looking LU with partial pivoting
  const int nb = R.nb;
  const int npan = (n + nb - 1) / nb;
  int* ipiv = (int*)dev_ensure(c, R.piv, (size_t)n * sizeof(int));
  char* Li = (char*)dev_ensure(c, R.Linv, (size_t)npan * nb * nb * es);
  char* Ui = (char*)dev_ensure(c, R.Uinv, (size_t)npan * nb * nb * es);
  for (int pi = 0; pi < npan; ++pi) {
    const int k0 = pi * nb, kb = std::min(nb, n - k0);
    std::vector<PanelTask> pt{PanelTask{Rm, Li + (size_t)pi * nb * nb * es, Ui + (size_t)pi * nb * nb * es, ipiv + k0,
                                        n, k0, k0, n - k0, kb}};
    const int i0 = c.st.add(pt);
    c.st.upload(c);
    {
      ProfScope ps(c, "root_panel", 8.0 * (n - k0) * (double)kb * kb / 2);
      ck(lu_panel(c.st.ptr<PanelTask>(i0), prec, (int*)c.statusbuf.p, c.stream), "root panel");
    }
    ck(swap_rows(Rm, n, ipiv + k0, k0, kb, 0, k0, prec, 0, c.stream), "root swaps left");
    ck(swap_rows(Rm, n, ipiv + k0, k0, kb, k0 + kb, n, prec, 0, c.stream), "root swaps right");
    c.launches += 3;
    c.stats.flops_factor += 8.0 * (n - k0) * (double)kb * kb / 2;
    const int rest = n - k0 - kb;
    if (rest > 0) {
      ApplyBatch ab;
      ab.add(Li + (size_t)pi * nb * nb * es, kb, OP_N, Rm + ((size_t)k0 + (size_t)(k0 + kb) * n) * es, n, kb, rest, 0);
      run_apply(c, ab, true, prec, "root trsm");
      GemmBatch g;
      g.task(Rm + ((size_t)(k0 + kb) + (size_t)(k0 + kb) * n) * es, n, rest, rest, -1.0, 1.0);
      g.pair(Rm + ((size_t)(k0 + kb) + (size_t)k0 * n) * es, n, OP_N, Rm + ((size_t)k0 + (size_t)(k0 + kb) * n) * es, n,
             OP_N, kb);
      g.close();
      run_gemm(c, g, prec, prec, prec, "root update");
      c.stats.flops_factor += ab.flops + g.flops;
    }
  }
}

void check_status(Ctx& c) {
  int st = 0;
  ck(cudaMemcpyAsync(&st, c.statusbuf.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "read status");
  ck(cudaStreamSynchronize(c.stream), "status sync");
  prof_resolve(c);
  if (st & 1) fail(H2_ESINGULAR, "zero pivot in a partial LU or in the final LU");
  if (st & 2) fail(H2_EINTERNAL, "Jacobi eigen-decomposition did not converge");
}

}  // namespace

void factorize(Ctx& c, double eps, int prec) {
  const auto t0 = std::chrono::steady_clock::now();
  c.factored = false;
  c.inverted = false;
  c.prec = prec;
  c.eps_fill = eps;
  c.stats.flops_factor = 0;
  prof_reset(c);
  const int64_t launches0 = c.launches;
  H2Host& H = c.H;
  const int L = H.L, l0 = H.l0;
  dev_ensure(c, c.statusbuf, 64);
  ck(cudaMemsetAsync(c.statusbuf.p, 0, 64, c.stream), "status memset");
  ck(cudaStreamSynchronize(c.stream), "sync");
  c.st.begin();
  if ((int)c.lev.size() != L - l0 + 1) {
    c.lev.clear();
    c.lev.resize(L - l0 + 1);
  }
  // leaf level: dense near blocks and leaf bases
  {
    std::vector<int> n(1 << L);
    for (int t = 0; t < (1 << L); ++t) n[t] = (int)H.tree.size[L][t];
    setup_level(c, c.lev[0], L, n, {});
    LevelF& F = c.lev[0];
    const size_t es = esz(prec);
    CopyBatch cb;
    for (size_t q = 0; q < F.near_pairs.size(); ++q) {
      const auto [a, b] = F.near_pairs[q];
      cb.add((const cd*)c.dD.p + c.D_off[q], P64, n[a], n[a], n[b], (char*)F.near_buf.p + F.near_off[q] * es, prec,
             n[a], n[a], n[b]);
    }
    for (int t = 0; t < (1 << L); ++t) {
      if (F.k0[t] > 0)
        cb.add((const cd*)c.dV.p + c.V_off[t], P64, n[t], n[t], F.k0[t], (cd*)F.B_buf.p + F.B_off[t], P64, n[t], n[t],
               F.k0[t]);
      if (n[t] > F.k0[t])
        cb.add((const cd*)c.dVp.p + c.Vp_off[t], P64, n[t], n[t], n[t] - F.k0[t], (cd*)F.Vp_buf.p + F.Vp_off[t], P64,
               n[t], n[t], n[t] - F.k0[t]);
    }
    run_copy(c, cb, "leaf init");
  }
  for (int li = 0; li <= L - l0; ++li) {
    LevelF& F = c.lev[li];
    c.prof_suffix = "@" + std::to_string(F.l);
    std::vector<char> done(F.nc, 0);
    for (const auto& bt : F.batches) process_batch(c, F, bt, done, eps);
    if (F.l > l0) merge_level(c, F, c.lev[li + 1]);
    else root_factor(c, F);
    check_status(c);
  }
  c.prof_suffix.clear();
  c.factored = true;
  c.stats.launches_factor = c.launches - launches0;
  c.stats.t_factor_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace h2
