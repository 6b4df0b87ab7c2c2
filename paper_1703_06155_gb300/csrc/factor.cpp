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
#include <memory>
#include <set>

#include "batch.h"

namespace h2 {
using namespace h2k;

void run_gemm(Ctx& c, GemmBatch& b, int pin, int pout, int pacc, const char* what) {
  if (b.empty()) return;
  HostScope hs(c, "run_gemm");
  const int pa = b.pina < 0 ? pin : b.pina;
  const int emul = (c.opts.gram_emulation && pa == P32 && pin == P32 && pacc == P64 && pout == P64) ? 1
                   : (c.mv_emul && pa == P64 && pin == P64 && pacc == P64 && pout == P64)   ? 2
                                                                                            : 0;
  const bool all32 = pa == P32 && pin == P32 && pacc == P32 && pout == P32;
  const int64_t ws = b.plan(c.opts.split_target > 0 ? c.opts.split_target : 8 * 152, pacc == P64, c.opts.tile_policy,
                            !emul, all32 && c.opts.tensor_cores == 2);
  if (b.tl.empty()) return;
  if (checks_on()) check_gemm(b, b.pina, pin, pout, what);
  void* wsp = nullptr;
  if (ws > 0) wsp = dev_ensure(c, c.gemm_ws, (size_t)ws * (pacc == P64 ? sizeof(cd) : sizeof(cf)));
  const int i0 = c.st.add(b.t), i1 = c.st.add(b.p), i2 = c.st.add(b.tl);
  c.st.upload(c);
  const int tc = ((b.shape == 0 || b.shape == 7) && all32) ? c.opts.tensor_cores : 0;
  const char* pipe = emul == 1      ? "fp32_df"
                     : emul == 2    ? "fp64_dd"
                     : pacc == P64  ? "fp64"
                     : tc == 2      ? "tcgen05_tf32x3"
                     : tc == 1      ? "mma_tf32x3"
                                    : "fp32";
  ProfScope ps(c, std::string("gemm:") + what, b.alg_flops, pipe);
  c.paths[std::string("gemm:") + pipe + ":" + std::to_string(h2k::gemm_tile_m(b.shape)) + "x" +
          std::to_string(h2k::gemm_tile_n(b.shape))]++;
  if (ws > 0) c.paths[std::string("gemm_splitk:") + pipe]++;
  ck(gemm(c.st.ptr<GemmTask>(i0), c.st.ptr<GemmPair>(i1), c.st.ptr<GemmTile>(i2), (int)b.tl.size(), pin, pout, pacc,
          wsp, c.stream, b.shape, b.pina, c.opts.tensor_cores, emul),
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
    ck(gemm_mirror(c.st.ptr<GemmTask>(i0), (int)b.t.size(), maxh, pout, h2k::gemm_tile_m(b.shape), c.stream), what);
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
  ProfScope ps(c, std::string(left ? "apply_left:" : "apply_right:") + what, b.flops, prec == P64 ? "fp64" : "fp32");
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
  HostScope hs(c, "run_copy");
  if (checks_on()) check_copy(b, what);
  const int i0 = c.st.add(b.t);
  c.st.upload(c);
  double bytes = 0, elems = 0;
  for (const CopyTask& t : b.t) {
    const double n = (double)t.rows * t.cols, ns = (double)std::min(t.rows, t.srows) * std::min(t.cols, t.scols);
    bytes += n * esz(t.dst_prec) * (t.mode == 1 ? 2 : 1) + (t.src ? ns * esz(t.src_prec) : 0.0);
    elems += n;
  }
  // CTAs per task for about 8K entries each: large blocks get enough CTAs
  // to keep many HBM requests in flight
  const int per = (int)std::min(32.0, std::max(1.0, std::ceil(elems / (double)b.t.size() / 8192.0)));
  ProfScope ps(c, std::string("copy:") + what, 0.0, nullptr, bytes);
  ck(copy2d(c.st.ptr<CopyTask>(i0), (int)b.t.size(), c.stream, per), what);
  c.launches++;
}

namespace {

void ensure_covered(Ctx& lc, Ctx& c, int ls);

// Step 2 / panel applications: in-place kernel or GEMM + copy (h2_opts.apply_path)
void run_apply_auto(Ctx& c, ApplyBatch& b, bool left, int prec, const char* what) {
  if (checks_on()) check_apply(b, left, prec, what);
  if (c.opts.apply_path == 1) run_apply(c, b, left, prec, what);
  else run_apply_gemm(c, b, left, prec, what);
}

void setup_level(Ctx& c, LevelF& F, int l, const std::vector<int>& n, const std::vector<Pair>& carried) {
  const H2Host& H = c.H;
  const int nc = 1 << l;
  {
    // keep the device arenas of an earlier factorization (grow-only)
    DevBuf b1 = std::move(F.near_buf), b4 = std::move(F.Q_buf), b5 = std::move(F.inv_buf), b6 = std::move(F.piv_buf),
           b7 = std::move(F.Ub_buf);
    F = LevelF();
    F.near_buf = std::move(b1);
    F.Q_buf = std::move(b4);
    F.inv_buf = std::move(b5);
    F.piv_buf = std::move(b6);
    F.Ub_buf = std::move(b7);
  }
  F.l = l;
  F.nc = nc;
  F.sym = c.fac_ldlt;
  F.n = n;
  F.k0 = H.rank[l];
  F.kt = F.k0;
  F.m.assign(nc, 0);
  F.nbrs = near_lists(H.part, l);
  if (c.opts.ordering == H2_ORDER_NATURAL) {
    for (int i = 0; i < nc; ++i) F.batches.push_back({i});
  } else {
    // the colouring depends on the partition only: computed once per level
    if ((int)c.colour_cache.size() <= l) c.colour_cache.resize(l + 1);
    if ((int)c.colour_cache[l].size() != nc) c.colour_cache[l] = greedy_colours(F.nbrs);
    const std::vector<int>& col = c.colour_cache[l];
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
  // block LDL^T: the stored block of the pair {a, b} is (min, max)
  auto alias_of = [&](const std::unordered_map<int64_t, int>& ids, int a, int b) {
    auto it = ids.find(pkey(b, a));
    if (it == ids.end()) fail(H2_EINTERNAL, "block LDL^T: pair without its transpose");
    return it->second;
  };
  F.near_off.assign(F.near_pairs.size(), 0);
  for (size_t q = 0; q < F.near_pairs.size(); ++q) {
    const auto [a, b] = F.near_pairs[q];
    F.near_id[pkey(a, b)] = (int)q;
    if (F.sym && a > b) continue;
    F.near_off[q] = tot;
    tot += (size_t)n[a] * n[b];
  }
  if (F.sym)
    for (size_t q = 0; q < F.near_pairs.size(); ++q) {
      const auto [a, b] = F.near_pairs[q];
      if (a > b) F.near_off[q] = F.near_off[alias_of(F.near_id, a, b)];
    }
  F.near_elems = tot;
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
    if (F.sym && a > b) continue;
    tot += (size_t)n[a] * n[b];
  }
  if (F.sym)
    for (size_t q = 0; q < F.fill_pairs.size(); ++q) {
      const auto [a, b] = F.fill_pairs[q];
      if (a > b) F.fill_off[q] = F.fill_off[alias_of(F.fill_id, a, b)];
    }
  F.fill_elems = tot;
  F.fill_row.assign(nc, {});
  F.fill_col.assign(nc, {});
  for (size_t q = 0; q < F.fill_pairs.size(); ++q) {
    F.fill_row[F.fill_pairs[q].first].push_back((int)q);
    F.fill_col[F.fill_pairs[q].second].push_back((int)q);
  }
  const int pp = l & 1;
  F.fill_ptr = (char*)dev_ensure(c, c.fill_pp[pp], tot * es);
  if (tot) ck(cudaMemsetAsync(F.fill_ptr, 0, tot * es, c.stream), "fill memset");
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
    ti += 2 * (size_t)n[i] * n[i];  // L^{-1}P, U^{-1}
    F.piv_off.push_back(tp);
    tp += n[i];
    F.Vp_off.push_back(tvp);
    tvp += (size_t)n[i] * (n[i] - F.k0[i]);
    F.voff[i] = F.vlen;
    F.vlen += n[i];
  }
  F.B_ptr = (cd*)dev_ensure(c, c.B_pp[pp], tb * sizeof(cd));
  dev_ensure(c, F.Q_buf, tq * es);
  dev_ensure(c, F.inv_buf, ti * es);
  dev_ensure(c, F.piv_buf, tp * sizeof(int));
  F.Vp_ptr = (cd*)dev_ensure(c, c.Vp_pp[pp], tvp * sizeof(cd));
  // sum of ||S||_F^2 over the admissible blocks of each row and column
  if ((int)c.snorm2_cache.size() <= l) c.snorm2_cache.resize(l + 1);
  std::vector<double>& sn = c.snorm2_cache[l];
  if ((int)sn.size() != nc) {
    sn.assign(nc, 0.0);
    for (size_t q = 0; q < H.part.adm[l].size(); ++q) {
      double v = 0;
      for (const cplx& z : H.S[l][q]) v += std::norm(z);
      sn[H.part.adm[l][q].first] += v;
      sn[H.part.adm[l][q].second] += v;
    }
  }
  F.snorm2 = sn;
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
  return Ptrs{(char*)F.near_buf.p, F.fill_ptr, F.B_ptr, (char*)F.Q_buf.p, (char*)F.inv_buf.p,
              (int*)F.piv_buf.p, esz(c.prec)};
}

// One elimination batch of one instance; a group of instances processes its
// jobs of the same level-from-leaf index and colour together.
struct Job {
  Ctx* c;
  LevelF* F;
  const std::vector<int>* bt;
  std::vector<char>* done;
};

// Step-0 data of one cluster (scratch offsets in its instance's scratch)
struct Info {
  int i, n, k0, p, rp = 0;
  bool fill;
  bool proj = false;  // Gram formed in complement coordinates: X = Vp^H F, G' = X X^H
  int64_t wsum = 0;   // total fill-in width of the row (and column)
  size_t M, T1, G, L, T, W, Qx, Z1, Gh, U, lam, W1, W2, Yf, Y1, X, tr, Vpf;
  std::vector<int> rowf, colf;
};

// All launches go to the stream and staging buffers of `lc`; every job's
// instance shares that stream.
void process_batches(Ctx& lc, std::vector<Job>& jobs, double eps) {
  const int prec = lc.prec;
  const size_t es = esz(prec);
  const size_t nj = jobs.size();
  std::vector<Ptrs> P(nj);
  std::vector<std::vector<Info>> info(nj);
  std::vector<cd*> S(nj);
  std::vector<int*> d_r(nj);
  auto NB = [&](size_t q, int j, int k) -> char* {
    const LevelF& F = *jobs[q].F;
    return P[q].near + F.near_off.at(F.near_id.at(pkey(j, k))) * es;
  };
  auto FB = [&](size_t q, int id) -> char* { return P[q].fill + jobs[q].F->fill_off[id] * es; };
  auto lo_of = [&](size_t q, int j) { return (*jobs[q].done)[j] ? jobs[q].F->m[j] : 0; };
  auto Vp = [&](size_t q, int i) { return jobs[q].F->Vp_ptr + jobs[q].F->Vp_off[i]; };
  // With a symmetric Z the column fill-ins are the transposed row fill-ins and
  // the column Gram equals the row Gram: only the row side is formed, and the
  // admissible-row norm is halved to match (the decisions are unchanged).
  auto snorm = [&](size_t q, int i) {
    return jobs[q].c->H.symmetric ? 0.5 * jobs[q].F->snorm2[i] : jobs[q].F->snorm2[i];
  };

  // ------------------------------ Phase A (FP64) ---------------------------
  // Vp: complement of the incoming basis (stored with the level); G' = Vp^H M
  // Vp is the Gram of eq. (16) in complement coordinates.
  bool anyfill = false;
  auto hsA = std::make_unique<HostScope>(lc, "phaseA-plan");
  for (size_t q = 0; q < nj; ++q) {
    Ctx& c = *jobs[q].c;
    LevelF& F = *jobs[q].F;
    P[q] = ptrs(c, F);
    size_t sc = 0;  // scratch in cd units
    for (int i : *jobs[q].bt) {
      Info f{};
      f.i = i;
      f.n = F.n[i];
      f.k0 = F.k0[i];
      f.p = f.n - f.k0;
      for (int id : F.fill_row[i])
        if (F.fill_live[id]) f.rowf.push_back(id);
      for (int id : F.fill_col[i])
        if (F.fill_live[id]) f.colf.push_back(id);
      f.fill = (!f.rowf.empty() || !f.colf.empty()) && f.p > 0;
      if (f.fill) {
        const size_t n = f.n, p = f.p;
        auto take = [&](size_t cnt) { const size_t o = sc; sc += cnt; return o; };
        for (int id : f.rowf) f.wsum += F.n[F.fill_pairs[id].second] - lo_of(q, F.fill_pairs[id].second);
        if (!c.H.symmetric)
          for (int id : f.colf) f.wsum += F.n[F.fill_pairs[id].first] - lo_of(q, F.fill_pairs[id].first);
        // Two ways to form G' = Vp^H M Vp (M = sum F F^H), FP64 flops:
        //   full:       M (4 n^2 W, Hermitian) + M Vp (8 n^2 p) + Vp^H (M Vp) (8 n p^2)
        //   projected:  X = Vp^H F (8 p n W) + X X^H (4 p^2 W, Hermitian)
        // With a complex64 bulk the fill-ins F carry FP32 rounding already, so
        // X is formed on the FP32 pipe (its singular values move by ~u32 ||F||,
        // the same order as that rounding) and only X X^H, the eigen-problem and
        // the rank decision run in FP64.  The FP64 bulk takes the cheaper order.
        const double W = (double)f.wsum, dn = n, dp = p;
        f.proj = prec == P32 ||
                 (8 * dp * dn + 4 * dp * dp) * W < 4 * dn * dn * W + 8 * dn * dn * dp + 8 * dn * dp * dp;
        f.tr = take(1);
        if (f.proj) {
          f.X = take(p * (size_t)f.wsum);
          // complex64 copy of Vp for the complex64 product X = Vp^H F (the
          // product rounds Vp to FP32 either way)
          if (prec == P32) f.Vpf = take((n * p + 1) / 2);
        } else {
          f.M = take(n * n);
          f.T1 = take(n * p);
        }
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
        anyfill = true;
      }
      info[q].push_back(f);
    }
    S[q] = (cd*)dev_ensure(c, c.scratch, (sc + 1) * sizeof(cd));
    const size_t nb = jobs[q].bt->size();
    d_r[q] = (int*)dev_ensure(c, c.normbuf, 3 * nb * sizeof(int) + 64);
    ck(cudaMemsetAsync(d_r[q], 0, 3 * nb * sizeof(int), lc.stream), "memset r");
  }
  std::vector<std::vector<int>> r(nj), sweeps(nj);
  size_t jac_rec = SIZE_MAX;
  bool heev_used = false;
  std::vector<std::pair<size_t, size_t>> eig_of;
  for (size_t q = 0; q < nj; ++q) r[q].assign(jobs[q].bt->size(), 0);
  hsA.reset();
  if (anyfill) {
    bool trace_forked = false;
    GemmBatch gM, gX, gXX, gT, gG;
    CopyBatch cvp;
    std::vector<PcholTask> pc;
    std::vector<FrobTask> ft;
    std::vector<FrobBlock> fb;
    int maxp = 0;
    for (size_t q = 0; q < nj; ++q) {
      const bool sym = jobs[q].c->H.symmetric;
      const LevelF& F = *jobs[q].F;
      for (size_t u = 0; u < info[q].size(); ++u) {
        Info& f = info[q][u];
        if (!f.fill) continue;
        const int n = f.n, p = f.p;
        cd* Sq = S[q];
        // trace(M) = sum of ||F||_F^2 over the row (and column) fill-ins
        const int b0 = (int)fb.size();
        // block LDL^T: a row fill-in (i, k), k < i, is the transposed stored
        // (k, i) and enters in the column form
        auto tr = [&](int k) { return F.sym && f.i > k; };
        for (int id : f.rowf) {
          const int k = F.fill_pairs[id].second, lo = lo_of(q, k);
          if (tr(k)) fb.push_back(FrobBlock{FB(q, id) + (size_t)lo * es, F.n[k], F.n[k] - lo, n});
          else fb.push_back(FrobBlock{FB(q, id) + (size_t)lo * n * es, n, n, F.n[k] - lo});
        }
        if (!sym)
          for (int id : f.colf) {
            const int k = F.fill_pairs[id].first, lo = lo_of(q, k);
            fb.push_back(FrobBlock{FB(q, id) + (size_t)lo * es, F.n[k], F.n[k] - lo, n});
          }
        ft.push_back(FrobTask{b0, (int)fb.size() - b0, (double*)(Sq + f.tr)});
        if (f.proj) {
          // X = Vp^H [F_row ..., F_col^T ...]  (p x W, bulk precision), then G' = X X^H
          int64_t off = 0;
          char* Xb = (char*)(Sq + f.X);
          const void* VA = Vp(q, f.i);
          if (prec == P32) {
            cvp.add(Vp(q, f.i), P64, n, n, p, Sq + f.Vpf, P32, n, n, p);
            VA = Sq + f.Vpf;
          }
          for (int id : f.rowf) {
            const int k = F.fill_pairs[id].second, lo = lo_of(q, k), w = F.n[k] - lo;
            gX.task(Xb + (size_t)off * p * es, p, p, w, 1.0, 0.0);
            if (tr(k)) gX.pair(VA, n, OP_H, FB(q, id) + (size_t)lo * es, F.n[k], OP_T, n);
            else gX.pair(VA, n, OP_H, FB(q, id) + (size_t)lo * n * es, n, OP_N, n);
            gX.close();
            off += w;
          }
          if (!sym)
            for (int id : f.colf) {
              const int k = F.fill_pairs[id].first, lo = lo_of(q, k), w = F.n[k] - lo;
              gX.task(Xb + (size_t)off * p * es, p, p, w, 1.0, 0.0);
              gX.pair(VA, n, OP_H, FB(q, id) + (size_t)lo * es, F.n[k], OP_T, n);
              gX.close();
              off += w;
            }
          if (prec == P32) {
            gXX.task(Sq + f.G, p, p, p, 1.0, 0.0);
            gXX.pair(Sq + f.X, p, OP_N, Sq + f.X, p, OP_H, (int)f.wsum);
            gXX.hermitian();
            gXX.close();
          } else {
            gG.task(Sq + f.G, p, p, p, 1.0, 0.0);
            gG.pair(Sq + f.X, p, OP_N, Sq + f.X, p, OP_H, (int)f.wsum);
            gG.hermitian();
            gG.close();
          }
        } else {
          gM.task(Sq + f.M, n, n, n, 1.0, 0.0);
          for (int id : f.rowf) {
            const int k = F.fill_pairs[id].second, lo = lo_of(q, k);
            if (tr(k)) {
              char* A = FB(q, id) + (size_t)lo * es;
              gM.pair(A, F.n[k], OP_T, A, F.n[k], OP_C, F.n[k] - lo);
            } else {
              char* A = FB(q, id) + (size_t)lo * n * es;
              gM.pair(A, n, OP_N, A, n, OP_H, F.n[k] - lo);
            }
          }
          if (!sym)
            for (int id : f.colf) {
              const int k = F.fill_pairs[id].first, lo = lo_of(q, k);
              char* A = FB(q, id) + (size_t)lo * es;
              gM.pair(A, F.n[k], OP_T, A, F.n[k], OP_C, F.n[k] - lo);
            }
          gM.hermitian();
          gM.close();
          gT.task(Sq + f.T1, n, n, p, 1.0, 0.0);
          gT.pair(Sq + f.M, n, OP_N, Vp(q, f.i), n, OP_N, n);
          gT.close();
          gG.task(Sq + f.G, p, p, p, 1.0, 0.0);
          gG.pair(Vp(q, f.i), n, OP_H, Sq + f.T1, n, OP_N, n);
          gG.close();
        }
        // the one-sided solver works on the Cholesky factor R, written into
        // the Ritz-matrix slot
        pc.push_back(PcholTask{Sq + f.G, (const double*)(Sq + f.tr), Sq + f.L, Sq + f.T, d_r[q] + u, p, n,
                               snorm(q, f.i), eps * eps, Sq + f.W, lc.opts.eig_solver == 2 ? Sq + f.Gh : nullptr,
                               prec == P32 ? 1 : 0});
        maxp = std::max(maxp, p);
      }
    }
    {
      const int i0 = lc.st.add(ft), i1 = lc.st.add(fb);
      lc.st.upload(lc);
      double tb = 0;
      for (const FrobBlock& f : fb) tb += (double)f.rows * f.cols * es;
      double* part = (double*)dev_ensure(lc, lc.frobbuf, (fb.size() + 1) * sizeof(double));
      if (lc.opts.profile == 0) {
        // the trace only reads the fill-ins: it runs on the side stream beside
        // the Gram products and joins before the subspace kernel reads it
        if (!lc.side.s) {
          ck(cudaStreamCreateWithFlags(&lc.side.s, cudaStreamNonBlocking), "side stream");
          ck(cudaEventCreateWithFlags(&lc.side.a, cudaEventDisableTiming), "side event");
          ck(cudaEventCreateWithFlags(&lc.side.b, cudaEventDisableTiming), "side event");
        }
        ck(cudaEventRecord(lc.side.a, lc.stream), "side fork");
        ck(cudaStreamWaitEvent(lc.side.s, lc.side.a, 0), "side fork");
        ck(frob2(lc.st.ptr<FrobTask>(i0), (int)ft.size(), lc.st.ptr<FrobBlock>(i1), (int)fb.size(), part, prec,
                 lc.side.s),
           "fill trace");
        ck(cudaEventRecord(lc.side.b, lc.side.s), "side join");
        trace_forked = true;
      } else {
        ProfScope ps(lc, "trace", 0.0, nullptr, tb);
        ck(frob2(lc.st.ptr<FrobTask>(i0), (int)ft.size(), lc.st.ptr<FrobBlock>(i1), (int)fb.size(), part, prec,
                 lc.stream),
           "fill trace");
      }
      lc.launches += 2;
    }
    run_gemm(lc, gM, prec, P64, P64, "gram");
    // X = Vp^H F: complex128 result with the FP64 bulk, complex64 (from the
    // complex64 copy of Vp, on the tensor cores) with the complex64 bulk; then
    // X X^H accumulates to FP64 accuracy
    run_copy(lc, cvp, "Vp to complex64");
    run_gemm(lc, gX, prec, prec, prec, "Vp^H*F");
    run_gemm(lc, gXX, P32, P64, P64, "X*X^H");
    run_gemm(lc, gT, P64, P64, P64, "gram*Vp");
    run_gemm(lc, gG, P64, P64, P64, "Vp^H*gram*Vp");
    size_t pchol_rec = SIZE_MAX;
    if (trace_forked) ck(cudaStreamWaitEvent(lc.stream, lc.side.b, 0), "side join");
    {
      const int i0 = lc.st.add(pc);
      lc.st.upload(lc);
      ProfScope ps(lc, "pchol_wy", 0.0, "fp64");
      if (ps.on) pchol_rec = ps.idx;
      int used = 0;
      ck(pchol_wy(lc.st.ptr<PcholTask>(i0), (int)pc.size(), maxp, lc.opts.cluster_max > 0 ? lc.opts.cluster_max : 16,
                  lc.stream, &used),
         "pivoted cholesky");
      lc.paths["pchol_wy:cta" + std::to_string(used)]++;
      lc.launches++;
    }
    std::vector<std::vector<int>> rp(nj);
    for (size_t q = 0; q < nj; ++q) {
      rp[q].assign(jobs[q].bt->size(), 0);
      ck(cudaMemcpyAsync(rp[q].data(), d_r[q], rp[q].size() * sizeof(int), cudaMemcpyDeviceToHost, lc.stream),
         "read r'");
    }
    sync_timed(lc, lc.stream, "sync after pivoted cholesky");
    lc.st.begin();
    for (size_t q = 0; q < nj; ++q)
      for (size_t u = 0; u < info[q].size(); ++u)
        if (info[q][u].fill) info[q][u].rp = std::min(std::max(rp[q][u], 0), info[q][u].p);
    if (pchol_rec != SIZE_MAX) {
      // algorithmic flops of the subspace kernel: pivoted Cholesky of the
      // p x p Gram to r' pivots (p r'^2 / 2 complex MACs), Householder QR of
      // the p x r' factor (2 p r'^2 - 2 r'^3 / 3) and its compact-WY T
      // (p r'^2 / 2); 8 real flops per complex MAC
      double fl = 0;
      for (size_t q = 0; q < nj; ++q)
        for (const Info& f : info[q])
          if (f.fill) {
            const double p = f.p, r = f.rp;
            fl += 8.0 * (p * r * r / 2 + 2 * p * r * r - 2 * r * r * r / 3 + p * r * r / 2);
          }
      lc.prof_open[pchol_rec].flops = fl;
    }
    // Ritz step on span(Qx) and the complement rotation Yf = Vp Q, Q = I - Y T Y^H
    GemmBatch g1, g2, g3, g4, g5;
    CopyBatch cp;
    std::vector<EigTask> eig;
    std::vector<SelTask> sel;
    int maxr = 0;
    for (size_t q = 0; q < nj; ++q)
      for (const Info& f : info[q])
        if (f.fill) maxr = std::max(maxr, f.rp);
    // one-sided Jacobi on R: no Ritz matrix (and no explicit Qx) is formed
    const bool use_osj = lc.opts.eig_solver == 2 && maxr <= osj_max_order();
    for (size_t q = 0; q < nj; ++q) {
      const size_t nb = jobs[q].bt->size();
      cd* Sq = S[q];
      for (size_t u = 0; u < info[q].size(); ++u) {
        Info& f = info[q][u];
        if (!f.fill || f.rp == 0) continue;
        const int n = f.n, p = f.p, rr = f.rp;
        cd* Y = Sq + f.L;
        g1.task(Sq + f.W, p, p, rr, 1.0, 0.0);  // W = Y T
        g1.pair(Y, p, OP_N, Sq + f.T, rr, OP_N, rr);
        g1.close();
        g1.task(Sq + f.W1, n, n, rr, 1.0, 0.0);  // W1 = Vp Y
        g1.pair(Vp(q, f.i), n, OP_N, Y, p, OP_N, p);
        g1.close();
        if (!use_osj) cp.add(nullptr, P64, p, 0, 0, Sq + f.Qx, P64, p, p, rr, 2);  // Qx = E
        cp.add(Vp(q, f.i), P64, n, n, p, Sq + f.Yf, P64, n, n, p, 0);                // Yf = Vp
        if (!use_osj) {
          g2.task(Sq + f.Qx, p, p, rr, -1.0, 1.0);  // Qx = E - W Y(0:r',:)^H
          g2.pair(Sq + f.W, p, OP_N, Y, p, OP_H, rr);
          g2.close();
        }
        g2.task(Sq + f.W2, n, n, rr, 1.0, 0.0);  // W2 = W1 T
        g2.pair(Sq + f.W1, n, OP_N, Sq + f.T, rr, OP_N, rr);
        g2.close();
        if (!use_osj) {
          g3.task(Sq + f.Z1, p, p, rr, 1.0, 0.0);  // Z1 = G' Qx
          g3.pair(Sq + f.G, p, OP_N, Sq + f.Qx, p, OP_N, p);
          g3.close();
        }
        g3.task(Sq + f.Yf, n, n, p, -1.0, 1.0);  // Yf = Vp - W2 Y^H
        g3.pair(Sq + f.W2, n, OP_N, Y, p, OP_H, rr);
        g3.close();
        if (!use_osj) {
          g4.task(Sq + f.Gh, rr, rr, rr, 1.0, 0.0);  // Ritz matrix Qx^H G' Qx
          g4.pair(Sq + f.Qx, p, OP_H, Sq + f.Z1, p, OP_N, p);
          g4.close();
        }
        // the Jacobi leaves entries below 1e-4 of the threshold unrotated: with
        // r' of them per row, the eigenvalues move by at most r' 1e-4 thr
        eig.push_back(EigTask{Sq + f.Gh, Sq + f.U, (double*)(Sq + f.lam), rr, d_r[q] + 2 * nb + u,
                              (const double*)(Sq + f.tr), snorm(q, f.i), eps * eps, 1e-4});
        eig_of.push_back({q, u});
        sel.push_back(
            SelTask{(const double*)(Sq + f.tr), (double*)(Sq + f.lam), d_r[q] + nb + u, n, rr, snorm(q, f.i), eps * eps});
        g5.task(Sq + f.Y1, n, n, rr, 1.0, 0.0);  // Y1 = Yf(:, 0:r') U
        g5.pair(Sq + f.Yf, n, OP_N, Sq + f.U, rr, OP_N, rr);
        g5.close();
      }
    }
    run_gemm(lc, g1, P64, P64, P64, "WY 1");
    run_copy(lc, cp, "WY presets");
    run_gemm(lc, g2, P64, P64, P64, "WY 2");
    run_gemm(lc, g3, P64, P64, P64, "WY 3");
    run_gemm(lc, g4, P64, P64, P64, "ritz matrix");
    const bool use_heev = lc.opts.eig_solver == 1 && maxr <= heev_max_order();
    if (!eig.empty() && use_osj) {
      const int i0 = lc.st.add(eig);
      lc.st.upload(lc);
      ProfScope ps(lc, "osj_cluster", 0.0, "fp32_dfr");
      if (ps.on) jac_rec = ps.idx;
      const int cmax = lc.opts.cluster_max > 0 ? lc.opts.cluster_max : 16;
      const int csize = osj_cluster_size((int)eig.size(), maxr, cmax);
      const int64_t per = osj_cluster_scratch(maxr);
      void* js = dev_ensure(lc, lc.jac_buf, (size_t)per * eig.size());
      int used = 0;
      ck(osj_eig_cluster(lc.st.ptr<EigTask>(i0), (int)eig.size(), maxr, csize, js, (int*)lc.statusbuf.p, lc.stream,
                         &used),
         "one-sided Jacobi (cluster)");
      lc.paths["osj_cluster:cta" + std::to_string(used)]++;
      lc.launches++;
      const int i1 = lc.st.add(sel);
      lc.st.upload(lc);
      ck(select_rank(lc.st.ptr<SelTask>(i1), (int)sel.size(), lc.stream), "select");
      lc.launches++;
    } else if (!eig.empty() && use_heev) {
      const int i0 = lc.st.add(eig);
      lc.st.upload(lc);
      ProfScope ps(lc, "heev_cluster", 0.0, "fp64");
      if (ps.on) jac_rec = ps.idx;
      heev_used = true;
      const int cmax = lc.opts.cluster_max > 0 ? lc.opts.cluster_max : 16;
      const int csize = heev_cluster_size((int)eig.size(), maxr, cmax);
      const int64_t per = heev_cluster_scratch(maxr);
      double* js = (double*)dev_ensure(lc, lc.jac_buf, (size_t)per * eig.size() * sizeof(double));
      int used = 0;
      ck(heev_cluster(lc.st.ptr<EigTask>(i0), (int)eig.size(), maxr, csize, js, (int*)lc.statusbuf.p, lc.stream,
                      &used),
         "tridiagonal QL eigen-decomposition");
      lc.paths["heev_cluster:cta" + std::to_string(used)]++;
      lc.launches++;
      const int i1 = lc.st.add(sel);
      lc.st.upload(lc);
      ck(select_rank(lc.st.ptr<SelTask>(i1), (int)sel.size(), lc.stream), "select");
      lc.launches++;
    } else if (!eig.empty()) {
      const int i0 = lc.st.add(eig);
      lc.st.upload(lc);
      ProfScope ps(lc, maxr >= 48 ? "jacobi_cluster" : "jacobi", 0.0, "fp64");
      if (ps.on) jac_rec = ps.idx;
      if (maxr >= 48) {
        // large Ritz problems: one cluster of CTAs per eigenproblem (16 when
        // few problems share the launch, so that more SMs work on each)
        const int64_t per = jacobi_cluster_scratch(maxr);
        double* js = (double*)dev_ensure(lc, lc.jac_buf, (size_t)per * eig.size() * sizeof(double));
        const int cmax = lc.opts.cluster_max > 0 ? lc.opts.cluster_max : 16;
        const int csize = std::min(cmax, eig.size() * 16 <= 152 ? 16 : 8);
        int used = 0;
        ck(jacobi_eig_cluster(lc.st.ptr<EigTask>(i0), (int)eig.size(), maxr, csize, js, (int*)lc.statusbuf.p,
                              lc.stream, &used),
           "jacobi (cluster)");
        lc.paths["jacobi_cluster:cta" + std::to_string(used)]++;
      } else {
        ck(jacobi_eig(lc.st.ptr<EigTask>(i0), (int)eig.size(), maxr, (int*)lc.statusbuf.p, lc.stream), "jacobi");
        lc.paths["jacobi:cta1"]++;
      }
      lc.launches++;
      const int i1 = lc.st.add(sel);
      lc.st.upload(lc);
      ck(select_rank(lc.st.ptr<SelTask>(i1), (int)sel.size(), lc.stream), "select");
      lc.launches++;
    }
    run_gemm(lc, g5, P64, P64, P64, "ritz vectors");
    for (size_t q = 0; q < nj; ++q) {
      const size_t nb = jobs[q].bt->size();
      sweeps[q].assign(nb, 0);
      ck(cudaMemcpyAsync(r[q].data(), d_r[q] + nb, nb * sizeof(int), cudaMemcpyDeviceToHost, lc.stream), "read r");
      ck(cudaMemcpyAsync(sweeps[q].data(), d_r[q] + 2 * nb, nb * sizeof(int), cudaMemcpyDeviceToHost, lc.stream),
         "read sweeps");
    }
  }
  sync_timed(lc, lc.stream, "sync after step 0");
  if (jac_rec != SIZE_MAX) {
    // algorithmic flops.  Hermitian Jacobi: 24 r'^3 real flops per sweep
    // (r'(r'-1)/2 complex rotations per sweep, each applied to two rows and
    // two columns of the r' x r' matrix and to two columns of U).
    // Tridiagonal path: (16/3) r'^3 (Householder reduction) + 8 r'^3
    // (back-transformation of r' vectors) + 3 r'^2 per QL sweep (a sweep's
    // rotations, r'/2 of them on average, applied to the r' rows of Z)
    double fl = 0;
    for (auto [q, u] : eig_of) {
      const double rr = info[q][u].rp;
      const double sw = std::max(sweeps[q][u], 0);
      // one-sided Jacobi: per sweep r'(r'-1)/2 pairs, each a complex dot
      // product of two columns of W (8 r' flops) and the rotation of two
      // columns of W and of J (20 r' flops each): 24 r'^3 per sweep as well
      fl += heev_used ? (16.0 / 3.0 + 8.0) * rr * rr * rr + 3.0 * rr * rr * sw : 24.0 * rr * rr * rr * sw;
    }
    lc.prof_open[jac_rec].flops = fl;
  }
  prof_resolve(lc);
  lc.st.begin();  // stream idle: staging can be reused
  for (size_t q = 0; q < nj; ++q) {
    LevelF& F = *jobs[q].F;
    for (size_t u = 0; u < info[q].size(); ++u) {
      const Info& f = info[q][u];
      const int rr = (f.fill && f.rp > 0) ? std::min(std::max(r[q][u], 0), f.rp) : 0;
      if (f.fill && f.rp > 0) {
        F.st_ritz_max = std::max(F.st_ritz_max, f.rp);
        F.st_ritz_sum += f.rp;
        F.st_ritz_n++;
        if (!sweeps[q].empty()) F.st_sweeps_max = std::max(F.st_sweeps_max, sweeps[q][u]);
      }
      r[q][u] = rr;
      F.kt[f.i] = f.k0 + rr;
      F.m[f.i] = f.n - F.kt[f.i];
    }
  }

  // ------------------------------ Phase B (bulk) ---------------------------
  auto hsB = std::make_unique<HostScope>(lc, "phaseB-Q-step2-plan");
  CopyBatch qc;
  for (size_t q = 0; q < nj; ++q) {
    const LevelF& F = *jobs[q].F;
    cd* Sq = S[q];
    for (size_t u = 0; u < info[q].size(); ++u) {
      const Info& f = info[q][u];
      const int n = f.n, m = F.m[f.i], rr = r[q][u];
      char* Q = P[q].Q + F.Q_off[f.i] * es;
      if (f.fill && f.rp > 0) {
        // Q~ = [Y1(:, r:r'), Yf(:, r':p), B, Y1(:, 0:r)]  (eqs. 18-19)
        const int rp = f.rp;
        qc.add(Sq + f.Y1 + (size_t)rr * n, P64, n, n, rp - rr, Q, prec, n, n, rp - rr);
        qc.add(Sq + f.Yf + (size_t)rp * n, P64, n, n, f.p - rp, Q + (size_t)(rp - rr) * n * es, prec, n, n, f.p - rp);
        if (rr > 0) qc.add(Sq + f.Y1, P64, n, n, rr, Q + (size_t)(m + f.k0) * n * es, prec, n, n, rr);
      } else {
        qc.add(Vp(q, f.i), P64, n, n, f.p, Q, prec, n, n, f.p);
      }
      qc.add(P[q].B + F.B_off[f.i], P64, n, n, f.k0, Q + (size_t)m * n * es, prec, n, n, f.k0);
    }
  }
  run_copy(lc, qc, "form Q");

  // Step 2: rows (left, Q^H) then columns (right, conj Q)
  ApplyBatch L2, R2;
  for (size_t q = 0; q < nj; ++q) {
    const LevelF& F = *jobs[q].F;
    for (int i : *jobs[q].bt) {
      const int n = F.n[i], m = F.m[i];
      const char* Q = P[q].Q + F.Q_off[i] * es;
      // block LDL^T: only the stored block of each pair is transformed; the
      // row transform of (i, j), j < i, is the column transform of (j, i)
      for (int j : F.nbrs[i]) {
        if (j == i) {
          L2.add(Q, n, OP_H, NB(q, i, i), n, n, n, 0);
          R2.add(Q, n, OP_C, NB(q, i, i), n, n, n, 0);
        } else {
          const int lo = lo_of(q, j);
          if (!F.sym || i < j) L2.add(Q, n, OP_H, NB(q, i, j) + (size_t)lo * n * es, n, n, F.n[j] - lo, 0);
          if (!F.sym || i > j) R2.add(Q, n, OP_C, NB(q, j, i) + (size_t)lo * es, F.n[j], n, F.n[j] - lo, 0);
        }
      }
      for (int id : F.fill_row[i]) {
        if (!F.fill_live[id]) continue;
        const int b = F.fill_pairs[id].second, lo = lo_of(q, b);
        if (F.sym && i > b) R2.add(Q, n, OP_C, FB(q, id) + (size_t)lo * es, F.n[b], n, F.n[b] - lo, m);
        else L2.add(Q, n, OP_H, FB(q, id) + (size_t)lo * n * es, n, n, F.n[b] - lo, m);
      }
      for (int id : F.fill_col[i]) {
        if (F.sym || !F.fill_live[id]) continue;
        const int a = F.fill_pairs[id].first, lo = lo_of(q, a);
        R2.add(Q, n, OP_C, FB(q, id) + (size_t)lo * es, F.n[a], n, F.n[a] - lo, m);
      }
    }
  }
  hsB.reset();
  run_apply_auto(lc, L2, true, prec, "step2 rows");
  run_apply_auto(lc, R2, false, prec, "step2 cols");
  const double f2 = (L2.flops + R2.flops) / (double)nj;

  // Step 3: LU + explicit inverses, panels, Schur
  std::vector<LuTask> lu;
  size_t lscr = 0;
  for (size_t q = 0; q < nj; ++q)
    for (int i : *jobs[q].bt)
      if (jobs[q].F->m[i] > 0) lscr += (size_t)jobs[q].F->n[i] * jobs[q].F->n[i];
  char* lsc = (char*)dev_ensure(lc, lc.lu_scr, (lscr + 1) * es);
  lscr = 0;
  for (size_t q = 0; q < nj; ++q) {
    const LevelF& F = *jobs[q].F;
    for (int i : *jobs[q].bt) {
      const int n = F.n[i], m = F.m[i];
      if (m <= 0) continue;
      char* inv = P[q].inv + F.inv_off[i] * es;
      lu.push_back(LuTask{NB(q, i, i), inv, inv + (size_t)n * n * es, P[q].piv + F.piv_off[i], n, m,
                          lsc + lscr * es});
      lscr += (size_t)n * n;
      jobs[q].c->stats.flops_factor += 8.0 / 3.0 * m * (double)m * m + 8.0 / 3.0 * m * (double)m * m;
    }
  }
  if (!lu.empty()) {
    if (checks_on()) check_lu(lu, prec);
    const int i0 = lc.st.add(lu);
    lc.st.upload(lc);
    double fl = 0;
    for (const LuTask& t : lu) fl += 16.0 / 3.0 * (double)t.m * t.m * t.m;
    ProfScope ps(lc, "lu", fl, prec == P64 ? "fp64" : "fp32");
    int maxm = 0;
    for (const LuTask& t : lu) maxm = std::max(maxm, t.m);
    ck(lu_blocked(lc.st.ptr<LuTask>(i0), (int)lu.size(), maxm, prec, (int*)lc.statusbuf.p, lc.stream), "lu");
    lc.launches++;
  }
  // Block LU: the panels L^{-1}P Z_i'c and Z_ci' U^{-1} in place (Alg. 4).
  // Block LDL^T (all jobs of a group share the form): the block row Z_i'c
  // stays raw, and W_ik = F^{-1} Z_i'k = U^{-1} (L^{-1}P Z_i'k) (a workspace;
  // the triangular factors applied in turn, as the LU panels apply them: a
  // product U^{-1} L^{-1}P formed first loses accuracy in complex64 where
  // the two factors cancel) is the right operand of the Schur updates
  // S_jk -= Z_ji' W_ik, formed for the stored pairs j <= k only.
  const bool sym = jobs[0].F->sym;
  double f3 = 0;
  std::vector<std::unordered_map<int64_t, size_t>> woff(nj);
  char* Wb = nullptr;
  if (sym) {
    GemmBatch gw;
    ApplyBatch pw;
    size_t wt = 0;
    for (size_t q = 0; q < nj; ++q) {
      const LevelF& F = *jobs[q].F;
      for (int i : *jobs[q].bt) {
        const int m = F.m[i];
        if (m <= 0) continue;
        for (int k : F.nbrs[i]) {
          const int clo = (k == i) ? m : lo_of(q, k);
          woff[q][pkey(i, k)] = wt;
          wt += (size_t)m * (F.n[k] - clo);
        }
      }
    }
    Wb = (char*)dev_ensure(lc, lc.ldlt_w, (wt + 1) * es);
    for (size_t q = 0; q < nj; ++q) {
      const LevelF& F = *jobs[q].F;
      for (int i : *jobs[q].bt) {
        const int n = F.n[i], m = F.m[i];
        if (m <= 0) continue;
        const char* Linv = P[q].inv + F.inv_off[i] * es;
        const char* Uinv = Linv + (size_t)n * n * es;
        for (int k : F.nbrs[i]) {
          const int clo = (k == i) ? m : lo_of(q, k);
          char* W = Wb + woff[q].at(pkey(i, k)) * es;
          gw.task(W, m, m, F.n[k] - clo, 1.0, 0.0);
          if (i > k)  // Z_i'k = rows clo.. of the stored (k, i), transposed
            gw.pair(Linv, m, OP_N, NB(q, i, k) + (size_t)clo * es, F.n[k], OP_T, m);
          else
            gw.pair(Linv, m, OP_N, NB(q, i, k) + (size_t)clo * n * es, n, OP_N, m);
          gw.close();
          pw.add(Uinv, m, OP_N, W, m, m, F.n[k] - clo, 0);
        }
      }
    }
    run_gemm(lc, gw, prec, prec, prec, "L^-1 Z");
    run_apply_auto(lc, pw, true, prec, "U^-1 W");
    f3 = (gw.flops + pw.flops) / (double)nj;
  } else {
    ApplyBatch PL, PR;
    for (size_t q = 0; q < nj; ++q) {
      const LevelF& F = *jobs[q].F;
      for (int i : *jobs[q].bt) {
        const int n = F.n[i], m = F.m[i];
        if (m <= 0) continue;
        const char* Linv = P[q].inv + F.inv_off[i] * es;
        const char* Uinv = Linv + (size_t)n * n * es;
        for (int j : F.nbrs[i]) {
          const int lo = (j == i) ? m : lo_of(q, j);
          PL.add(Linv, m, OP_N, NB(q, i, j) + (size_t)lo * n * es, n, m, F.n[j] - lo, 0);
          PR.add(Uinv, m, OP_N, NB(q, j, i) + (size_t)lo * es, F.n[j], m, F.n[j] - lo, 0);
        }
      }
    }
    run_apply_auto(lc, PL, true, prec, "U panels");
    run_apply_auto(lc, PR, false, prec, "L panels");
    f3 = (PL.flops + PR.flops) / (double)nj;
  }

  GemmBatch gs;
  auto hsS = std::make_unique<HostScope>(lc, "schur-plan");
  for (size_t q = 0; q < nj; ++q) {
    LevelF& F = *jobs[q].F;
    const std::vector<int>& bt = *jobs[q].bt;
    std::vector<char> inb(F.nc, 0);
    for (int i : bt) inb[i] = 1;
    // (target block (j, k), eliminated cluster i) for every i of the batch and
    // j, k in its near list, grouped by target in increasing key order (the
    // clusters of one target in batch order)
    std::vector<std::pair<int64_t, int>> tgl;
    for (int i : bt) {
      if (F.m[i] <= 0) continue;
      for (int j : F.nbrs[i])
        for (int k : F.nbrs[i])
          if (!sym || j <= k) tgl.emplace_back(pkey(j, k), i);
    }
    std::stable_sort(tgl.begin(), tgl.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    const double fl0 = gs.flops;
    for (size_t g0 = 0; g0 < tgl.size();) {
      size_t g1 = g0;
      while (g1 < tgl.size() && tgl[g1].first == tgl[g0].first) ++g1;
      const int64_t key = tgl[g0].first;
      const int j = (int)(key >> 32), k = (int)(uint32_t)key;
      const int rlo = inb[j] ? F.m[j] : lo_of(q, j);
      const int clo = inb[k] ? F.m[k] : lo_of(q, k);
      const int nj_ = F.n[j], nk = F.n[k];
      char* C;
      auto it = F.near_id.find(key);
      if (it != F.near_id.end()) {
        C = P[q].near + F.near_off[it->second] * es;
      } else {
        const int id = F.fill_id.at(key);
        C = FB(q, id);
        F.fill_live[id] = 1;
        if (sym) F.fill_live[F.fill_id.at(pkey(k, j))] = 1;
      }
      gs.task(C + ((size_t)rlo + (size_t)clo * nj_) * es, nj_, nj_ - rlo, nk - clo, -1.0, 1.0);
      for (size_t u = g0; u < g1; ++u) {
        const int i = tgl[u].second;
        const int ni = F.n[i], mi = F.m[i];
        if (!sym) {
          gs.pair(NB(q, j, i) + (size_t)rlo * es, nj_, OP_N, NB(q, i, k) + (size_t)clo * ni * es, ni, OP_N, mi);
        } else {
          // Z_ji' = rows rlo.. of the logical (j, i): the stored (i, j) transposed when j > i
          const char* W = Wb + woff[q].at(pkey(i, k)) * es;
          if (j > i) gs.pair(NB(q, i, j) + (size_t)rlo * ni * es, ni, OP_T, W, mi, OP_N, mi);
          else gs.pair(NB(q, j, i) + (size_t)rlo * es, nj_, OP_N, W, mi, OP_N, mi);
        }
      }
      gs.close();
      g0 = g1;
    }
    jobs[q].c->stats.flops_factor += gs.flops - fl0 + f2 + f3;
  }
  hsS.reset();
  run_gemm(lc, gs, prec, prec, prec, "schur");
  for (size_t q = 0; q < nj; ++q)
    for (int i : *jobs[q].bt) (*jobs[q].done)[i] = 1;
}

// Sets up the parent level and appends its merge copies to `as` / `ac` (the
// caller launches them, for all instances of a group at once).
void merge_level(Ctx& c, LevelF& F, LevelF& Pn, CopyBatch& as, CopyBatch& ac) {
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
  // kept part of the level's block (a, b) into dst (kt_a x kt_b, leading
  // dimension ld), assigned or accumulated; block LDL^T: (a, b), a > b, is
  // the stored (b, a) transposed
  auto kept_copy = [&](CopyBatch& cb, const char* base, size_t off, int a, int b, char* d, int ld, int mode) {
    if (F.sym && a > b) {
      cb.add(base + (off + (size_t)F.m[b] + (size_t)F.m[a] * F.n[b]) * es, prec, F.n[b], F.kt[a], F.kt[b], d, prec,
             ld, F.kt[a], F.kt[b], mode);
      cb.t.back().transpose = 1;
    } else {
      cb.add(base + (off + (size_t)F.m[a] + (size_t)F.m[b] * F.n[a]) * es, prec, F.n[a], F.kt[a], F.kt[b], d, prec,
             ld, F.kt[a], F.kt[b], mode);
    }
  };
  for (size_t q = 0; q < Pn.near_pairs.size(); ++q) {
    const auto [p, r] = Pn.near_pairs[q];
    if (Pn.sym && p > r) continue;
    char* dst = D.near + Pn.near_off[q] * es;
    const int ld = Pn.n[p];
    for (int a = 2 * p; a <= 2 * p + 1; ++a)
      for (int b = 2 * r; b <= 2 * r + 1; ++b) {
        char* d = dst + ((size_t)ro(a) + (size_t)ro(b) * ld) * es;
        const int64_t key = pkey(a, b);
        if (F.near_id.count(key)) {
          kept_copy(as, S.near, F.near_off[F.near_id.at(key)], a, b, d, ld, 0);
        } else {
          const int idx = c.adm_id[l].at(key);
          as.add((char*)c.dS.p + c.S_off[l][idx] * sizeof(cd), P64, F.k0[a], F.k0[a], F.k0[b], d, prec, ld, F.kt[a],
                 F.kt[b]);
          auto it = F.fill_id.find(key);
          if (it != F.fill_id.end() && F.fill_live[it->second])
            kept_copy(ac, S.fill, F.fill_off[it->second], a, b, d, ld, 1);
        }
      }
  }
  for (size_t q = 0; q < F.fill_pairs.size(); ++q) {
    if (!F.fill_live[q] || F.fill_is_adm[q]) continue;
    const auto [a, b] = F.fill_pairs[q];
    if (F.sym && a > b) continue;  // the stored (b, a) carries it
    if (F.sym && a / 2 == b / 2) fail(H2_EINTERNAL, "block LDL^T: pushed fill-in between siblings");
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
    cd* V = Pn.Vp_ptr + Pn.Vp_off[p];
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
}

// Blocked right-looking LU with partial pivoting of the final block of every
// instance (Algorithm 1, last line); panel step pi of all instances runs in
// the same launches.
void root_factor_group(Ctx& lc, const std::vector<Ctx*>& cs) {
  const int prec = lc.prec;
  const size_t es = esz(prec);
  CopyBatch as, ac;
  int npan_max = 0;
  for (Ctx* cp : cs) ensure_covered(lc, *cp, cp->lev.back().l);
  for (Ctx* cp : cs) {
    Ctx& c = *cp;
    LevelF& F = c.lev.back();
    const int l = F.l;
    RootF& R = c.root;
    R.kt = F.kt;
    std::vector<int> off(F.nc + 1, 0);
    for (int a = 0; a < F.nc; ++a) off[a + 1] = off[a] + F.kt[a];
    const int n = off[F.nc];
    R.n = n;
    if (n == 0) continue;
    char* Rm = (char*)dev_ensure(c, R.R, (size_t)n * n * es);
    Ptrs S = ptrs(c, F);
    for (int a = 0; a < F.nc; ++a)
      for (int b = 0; b < F.nc; ++b) {
        char* d = Rm + ((size_t)off[a] + (size_t)off[b] * n) * es;
        const int64_t key = pkey(a, b);
        // kept part of (a, b); block LDL^T: (a, b), a > b, is the stored (b, a) transposed
        auto kept_copy = [&](CopyBatch& cb, const char* base, size_t o, int mode) {
          if (F.sym && a > b) {
            cb.add(base + (o + (size_t)F.m[b] + (size_t)F.m[a] * F.n[b]) * es, prec, F.n[b], F.kt[a], F.kt[b], d,
                   prec, n, F.kt[a], F.kt[b], mode);
            cb.t.back().transpose = 1;
          } else {
            cb.add(base + (o + (size_t)F.m[a] + (size_t)F.m[b] * F.n[a]) * es, prec, F.n[a], F.kt[a], F.kt[b], d,
                   prec, n, F.kt[a], F.kt[b], mode);
          }
        };
        if (F.near_id.count(key)) {
          kept_copy(as, S.near, F.near_off[F.near_id.at(key)], 0);
        } else {
          auto ai = c.adm_id[l].find(key);
          if (ai != c.adm_id[l].end()) {
            as.add((char*)c.dS.p + c.S_off[l][ai->second] * sizeof(cd), P64, F.k0[a], F.k0[a], F.k0[b], d, prec, n,
                   F.kt[a], F.kt[b]);
          } else {
            // early stop: the pair lies inside an ancestor's admissible block
            auto ci = c.cov_off.find(key);
            if (c.cov_level != l || ci == c.cov_off.end())
              fail(H2_EINTERNAL, "final block: pair neither near nor admissible");
            as.add((char*)c.cov_buf.p + ci->second * sizeof(cd), P64, F.k0[a], F.k0[a], F.k0[b], d, prec, n,
                   F.kt[a], F.kt[b]);
          }
          auto it = F.fill_id.find(key);
          if (it != F.fill_id.end() && F.fill_live[it->second]) kept_copy(ac, S.fill, F.fill_off[it->second], 1);
        }
      }
    const int nb = R.nb;
    const int npan = (n + nb - 1) / nb;
    dev_ensure(c, R.piv, (size_t)n * sizeof(int));
    dev_ensure(c, R.Linv, (size_t)npan * nb * nb * es);
    dev_ensure(c, R.Uinv, (size_t)npan * nb * nb * es);
    npan_max = std::max(npan_max, npan);
  }
  run_copy(lc, as, "root assemble");
  run_copy(lc, ac, "root assemble fill");
  for (int pi = 0; pi < npan_max; ++pi) {
    std::vector<PanelTask> pt;
    std::vector<SwapTask> sw;
    ApplyBatch ab;
    GemmBatch g;
    double fl = 0;
    int maxrows = 0, maxkb = 0;
    for (Ctx* cp : cs) {
      Ctx& c = *cp;
      RootF& R = c.root;
      const int n = R.n, nb = R.nb;
      if (pi * nb >= n) continue;
      char* Rm = (char*)R.R.p;
      char* Li = (char*)R.Linv.p;
      char* Ui = (char*)R.Uinv.p;
      int* ipiv = (int*)R.piv.p;
      const int k0 = pi * nb, kb = std::min(nb, n - k0);
      pt.push_back(PanelTask{Rm, Li + (size_t)pi * nb * nb * es, Ui + (size_t)pi * nb * nb * es, ipiv + k0, n, k0, k0,
                             n - k0, kb});
      maxrows = std::max(maxrows, n - k0);
      maxkb = std::max(maxkb, kb);
      sw.push_back(SwapTask{Rm, ipiv + k0, n, k0, kb, 0, k0, 0});
      sw.push_back(SwapTask{Rm, ipiv + k0, n, k0, kb, k0 + kb, n, 0});
      c.stats.flops_factor += 8.0 * (n - k0) * (double)kb * kb / 2;
      fl += 8.0 * (n - k0) * (double)kb * kb / 2;
      const int rest = n - k0 - kb;
      if (rest > 0) {
        const double f0 = g.flops, a0 = ab.flops;
        ab.add(Li + (size_t)pi * nb * nb * es, kb, OP_N, Rm + ((size_t)k0 + (size_t)(k0 + kb) * n) * es, n, kb, rest, 0);
        g.task(Rm + ((size_t)(k0 + kb) + (size_t)(k0 + kb) * n) * es, n, rest, rest, -1.0, 1.0);
        g.pair(Rm + ((size_t)(k0 + kb) + (size_t)k0 * n) * es, n, OP_N, Rm + ((size_t)k0 + (size_t)(k0 + kb) * n) * es,
               n, OP_N, kb);
        g.close();
        c.stats.flops_factor += g.flops - f0 + ab.flops - a0;
      }
    }
    {
      const int i0 = lc.st.add(pt), i1 = lc.st.add(sw);
      lc.st.upload(lc);
      {
        ProfScope ps(lc, "root_panel", fl, prec == P64 ? "fp64" : "fp32");
        ck(lu_panel(lc.st.ptr<PanelTask>(i0), (int)pt.size(), prec, maxrows, maxkb, (int*)lc.statusbuf.p, lc.stream),
           "root panel");
      }
      ck(swap_rows_batch(lc.st.ptr<SwapTask>(i1), (int)sw.size(), prec, lc.stream), "root swaps");
      lc.launches += 2;
    }
    run_apply(lc, ab, true, prec, "root trsm");
    run_gemm(lc, g, prec, prec, prec, "root update");
  }
}

// Explicit inverse of every instance's final block (R^{-1} = the blocked LU
// solve applied to the identity), so that a solve's final-block step is one
// GEMM (the paper's eq. 35 inverse of the last factor).
void root_inverse_group(Ctx& lc, const std::vector<Ctx*>& cs) {
  const int prec = lc.prec;
  const size_t es = esz(prec);
  std::vector<char*> xs;
  std::vector<int> lds;
  std::vector<Ctx*> act;
  for (Ctx* c : cs) {
    const int n = c->root.n;
    if (n == 0) continue;
    char* Ri = (char*)dev_ensure(*c, c->root.Rinv, (size_t)n * n * es);
    ck(cudaMemsetAsync(Ri, 0, (size_t)n * n * es, lc.stream), "Rinv memset");
    ck(set_diag(Ri, n, n, prec, 1.0, lc.stream), "Rinv identity");
    lc.launches++;
    xs.push_back(Ri);
    lds.push_back(n);
    act.push_back(c);
  }
  if (act.empty()) return;
  // the RHS widths differ per instance: group by width
  std::map<int, std::vector<size_t>> by;
  for (size_t q = 0; q < act.size(); ++q) by[act[q]->root.n].push_back(q);
  for (auto& [n, qs] : by) {
    std::vector<Ctx*> c2;
    std::vector<char*> x2;
    std::vector<int> l2;
    for (size_t q : qs) {
      c2.push_back(act[q]);
      x2.push_back(xs[q]);
      l2.push_back(lds[q]);
    }
    root_solve_grouped(lc, c2, x2, l2, n, false);
  }
}

// The last factorized level: l0, or the early-stop level of the options.
int stop_of(const Ctx& c) {
  const int l0 = c.H.l0, L = c.H.L;
  return c.opts.stop_level > 0 ? std::max(l0, std::min(L, c.opts.stop_level)) : l0;
}

// Couplings of the pairs (a, b) of level ls > l0 that lie inside the
// admissible block (A, B) of an ancestor level lv: in the level-ls bases of a
// and b they are E_a S_AB E_b^T, where V_A(rows of a) = V_a E_a and E_a is the
// product of the transfer blocks on the path from a up to A (eq. 3).  They
// depend on the H^2 matrix only and are kept until it changes.  Launches go
// to lc's stream; the buffers belong to c.
void ensure_covered(Ctx& lc, Ctx& c, int ls) {
  const H2Host& H = c.H;
  const int l0 = H.l0;
  if (ls <= l0 || c.cov_level == ls) return;
  const int nc = 1 << ls;
  const std::vector<int>& kl = H.rank[ls];
  std::vector<std::vector<size_t>> eoff(nc, std::vector<size_t>(ls, 0));
  size_t etot = 0;
  for (int a = 0; a < nc; ++a)
    for (int lv = ls - 1; lv >= l0; --lv) {
      eoff[a][lv] = etot;
      etot += (size_t)kl[a] * H.rank[lv][a >> (ls - lv)];
    }
  cd* E = (cd*)dev_ensure(c, c.cov_E, (etot + 1) * sizeof(cd));
  const cd* T = (const cd*)c.dT.p;
  auto tslice = [&](int lv, int child) {  // rows of `child` (level lv+1) in the transfer of its parent
    const int p = child >> 1, k1 = H.rank[lv + 1][2 * p];
    return T + c.T_off[lv][p] + ((child & 1) ? k1 : 0);
  };
  auto tld = [&](int lv, int child) { const int p = child >> 1; return H.rank[lv + 1][2 * p] + H.rank[lv + 1][2 * p + 1]; };
  {
    CopyBatch cb;
    for (int a = 0; a < nc; ++a) {
      const int kp = H.rank[ls - 1][a >> 1];
      cb.add(tslice(ls - 1, a), P64, tld(ls - 1, a), kl[a], kp, E + eoff[a][ls - 1], P64, kl[a], kl[a], kp);
    }
    run_copy(lc, cb, "ancestor maps");
  }
  for (int lv = ls - 2; lv >= l0; --lv) {
    GemmBatch g;
    for (int a = 0; a < nc; ++a) {
      const int c1 = a >> (ls - lv - 1), kc = H.rank[lv + 1][c1], kp = H.rank[lv][c1 >> 1];
      g.task(E + eoff[a][lv], kl[a], kl[a], kp, 1.0, 0.0);
      g.pair(E + eoff[a][lv + 1], kl[a], OP_N, tslice(lv, c1), tld(lv, c1), OP_N, kc);
      g.close();
    }
    run_gemm(lc, g, P64, P64, P64, "ancestor maps");
  }
  std::set<Pair> near(H.part.inad[ls].begin(), H.part.inad[ls].end());
  struct Cov { int a, b, lv, q; };
  std::vector<Cov> cov;
  for (int a = 0; a < nc; ++a)
    for (int b = 0; b < nc; ++b) {
      if (near.count({a, b}) || c.adm_id[ls].count(pkey(a, b))) continue;
      int found = -1, q = -1;
      for (int lv = ls - 1; lv >= l0 && found < 0; --lv) {
        auto it = c.adm_id[lv].find(pkey(a >> (ls - lv), b >> (ls - lv)));
        if (it != c.adm_id[lv].end()) { found = lv; q = it->second; }
      }
      if (found < 0) fail(H2_EINTERNAL, "early stop: a level pair lies in no block of the partition");
      cov.push_back(Cov{a, b, found, q});
    }
  size_t ytot = 0, stot = 0;
  std::vector<size_t> yoff(cov.size());
  c.cov_off.clear();
  for (size_t u = 0; u < cov.size(); ++u) {
    const Cov& v = cov[u];
    yoff[u] = ytot;
    ytot += (size_t)kl[v.a] * H.rank[v.lv][v.b >> (ls - v.lv)];
    c.cov_off[pkey(v.a, v.b)] = stot;
    stot += (size_t)kl[v.a] * kl[v.b];
  }
  cd* Y = (cd*)dev_ensure(c, c.cov_Y, (ytot + 1) * sizeof(cd));
  cd* S = (cd*)dev_ensure(c, c.cov_buf, (stot + 1) * sizeof(cd));
  GemmBatch g1, g2;
  for (size_t u = 0; u < cov.size(); ++u) {
    const Cov& v = cov[u];
    const int A = v.a >> (ls - v.lv), B = v.b >> (ls - v.lv);
    const int kA = H.rank[v.lv][A], kB = H.rank[v.lv][B], ka = kl[v.a], kb = kl[v.b];
    g1.task(Y + yoff[u], ka, ka, kB, 1.0, 0.0);  // Y = E_a S_AB
    g1.pair(E + eoff[v.a][v.lv], ka, OP_N, (const cd*)c.dS.p + c.S_off[v.lv][v.q], kA, OP_N, kA);
    g1.close();
    g2.task(S + c.cov_off[pkey(v.a, v.b)], ka, ka, kb, 1.0, 0.0);  // Y E_b^T
    g2.pair(Y + yoff[u], ka, OP_N, E + eoff[v.b][v.lv], kb, OP_T, kB);
    g2.close();
  }
  run_gemm(lc, g1, P64, P64, P64, "ancestor couplings");
  run_gemm(lc, g2, P64, P64, P64, "ancestor couplings");
  c.cov_level = ls;
}

void check_status(Ctx& c) {
  int st = 0;
  ck(cudaMemcpyAsync(&st, c.statusbuf.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "read status");
  sync_timed(c, c.stream, "status sync");
  prof_resolve(c);
  if (st & 1) fail(H2_ESINGULAR, "zero pivot in a partial LU or in the final LU");
  if (st & 2) fail(H2_EINTERNAL, "Jacobi eigen-decomposition did not converge");
  if (c.opts.tensor_cores == 2 && h2k::gemm_umma_timeouts() != 0)
    fail(H2_ETIMEOUT, "a tensor-core GEMM tile gave up waiting for its MMAs (bounded mbarrier wait)");
}

}  // namespace

// Algorithm 1 for a group of independent instances: level-from-leaf index
// d and colour b of every instance run in the same launches (instances of
// different depth join as their levels come up).  All launches go to the
// first instance's stream; the others' streams are set to it for the call.
void factorize_group(const std::vector<Ctx*>& cs, double eps, int prec) {
  const auto t0 = std::chrono::steady_clock::now();
  Ctx& lc = *cs[0];
  // block LDL^T (h2_opts.ldlt: 1, or 2 for an FP64 factorization) when every
  // instance asks for it and is complex symmetric (the launches of a group
  // share one form), else block LU
  bool ldlt = true;
  for (Ctx* c : cs)
    ldlt = ldlt && (c->opts.ldlt == 1 || (c->opts.ldlt == 2 && prec == P64)) && c->H.symmetric;
  for (Ctx* c : cs) {
    c->fac_ldlt = ldlt;
    c->stream = lc.stream;
    c->epoch++;
    c->factored = false;
    c->inverted = false;
    c->prec = prec;
    c->eps_fill = eps;
    c->stats.flops_factor = 0;
    c->stats.t_sync_ms = 0;
    prof_reset(*c);
  }
  const int64_t launches0 = lc.launches;
  dev_ensure(lc, lc.statusbuf, 64);
  ck(cudaMemsetAsync(lc.statusbuf.p, 0, 64, lc.stream), "status memset");
  ck(cudaStreamSynchronize(lc.stream), "sync");
  lc.st.begin();
  int depth = 0;  // levels L .. (l0 or the stop level) of the deepest instance
  {
    CopyBatch cb;
    for (Ctx* cp : cs) {
      Ctx& c = *cp;
      H2Host& H = c.H;
      const int L = H.L, l0 = stop_of(c);
      depth = std::max(depth, L - l0 + 1);
      if ((int)c.lev.size() != L - l0 + 1) {
        for (LevelF& F : c.lev)
          for (DevBuf* b : {&F.near_buf, &F.Q_buf, &F.inv_buf, &F.piv_buf, &F.Ub_buf}) dev_free(c, *b);
        c.lev.clear();
        c.lev.resize(L - l0 + 1);
      }
      c.stats.stop_level = l0;
      // leaf level: dense near blocks and leaf bases
      std::vector<int> n(1 << L);
      for (int t = 0; t < (1 << L); ++t) n[t] = (int)H.tree.size[L][t];
      setup_level(c, c.lev[0], L, n, {});
      LevelF& F = c.lev[0];
      const size_t es = esz(prec);
      for (size_t q = 0; q < F.near_pairs.size(); ++q) {
        const auto [a, b] = F.near_pairs[q];
        if (F.sym && a > b) continue;
        cb.add((const cd*)c.dD.p + c.D_off[q], P64, n[a], n[a], n[b], (char*)F.near_buf.p + F.near_off[q] * es, prec,
               n[a], n[a], n[b]);
      }
      for (int t = 0; t < (1 << L); ++t) {
        if (F.k0[t] > 0)
          cb.add((const cd*)c.dV.p + c.V_off[t], P64, n[t], n[t], F.k0[t], F.B_ptr + F.B_off[t], P64, n[t],
                 n[t], F.k0[t]);
        if (n[t] > F.k0[t])
          cb.add((const cd*)c.dVp.p + c.Vp_off[t], P64, n[t], n[t], n[t] - F.k0[t], F.Vp_ptr + F.Vp_off[t], P64,
                 n[t], n[t], n[t] - F.k0[t]);
      }
    }
    run_copy(lc, cb, "leaf init");
  }
  for (int d = 0; d < depth; ++d) {
    std::vector<Ctx*> act;
    for (Ctx* c : cs)
      if (d < (int)c->lev.size()) act.push_back(c);
    lc.prof_suffix = "@d" + std::to_string(d);
    if (cs.size() == 1) lc.prof_suffix = "@" + std::to_string(cs[0]->lev[d].l);
    std::vector<std::vector<char>> done(act.size());
    size_t nbat = 0;
    for (size_t q = 0; q < act.size(); ++q) {
      done[q].assign(act[q]->lev[d].nc, 0);
      nbat = std::max(nbat, act[q]->lev[d].batches.size());
    }
    for (size_t b = 0; b < nbat; ++b) {
      std::vector<Job> jobs;
      for (size_t q = 0; q < act.size(); ++q) {
        LevelF& F = act[q]->lev[d];
        if (b < F.batches.size()) jobs.push_back(Job{act[q], &F, &F.batches[b], &done[q]});
      }
      process_batches(lc, jobs, eps);
    }
    CopyBatch as, ac;
    std::vector<Ctx*> roots;
    auto hsM = std::make_unique<HostScope>(lc, "merge-setup");
    for (Ctx* c : act) {
      if (d + 1 < (int)c->lev.size()) merge_level(*c, c->lev[d], c->lev[d + 1], as, ac);
      else roots.push_back(c);
    }
    hsM.reset();
    run_copy(lc, as, "merge");
    run_copy(lc, ac, "merge fill");
    if (!roots.empty()) {
      root_factor_group(lc, roots);
      root_inverse_group(lc, roots);
    }
    check_status(lc);
  }
  lc.prof_suffix.clear();
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (Ctx* c : cs) {
    c->factored = true;
    c->stats.t_factor_ms = ms;
  }
  lc.stats.launches_factor = lc.launches - launches0;
}

void factorize(Ctx& c, double eps, int prec) { factorize_group({&c}, eps, prec); }

}  // namespace h2
