// h2_build: H^2 representation of Z = I + s D^{1/2} K D^{1/2} by nested
// interpolative decompositions of exact far-field samples.
//
// The paper builds its H^2 matrices with the method of its refs. [14], [15]
// and does not describe it (Sec. VI).  This construction, for each level from
// the leaves up and each cluster t:
//   rows_t   the points of t (leaf) or the skeletons of its two children
//   sample   Z(rows_t, F*(t)), F*(t) = every point of the clusters admissible
//            with t or with an ancestor of t (all of t's far field); only its
//            Gram G_t = Z Z^H is formed (GPU kernel, O(N^2 k) FP64 work)
//   ID       pivoted Cholesky of G_t (the column-pivoted QR of Z^H in Gram
//            form): pivot = largest remaining diagonal, stop when it is
//            <= eps^2 times the first; the pivots are the skeleton rows and
//            P_t = L(rest) L(skel)^{-1} interpolates the others, so that
//            Z(rows_t, F*) ~= P_t Z(skel_t, F*)
//   basis    P_t = Q R (leaf: V_t = Q) or diag(R_t1, R_t2) P_t = Q R
//            (non-leaf: T_t = Q), so the bases are orthonormal and nested
//            (eq. 3); couplings S_ts = R_t Z(skel_t, skel_s) R_s^T (eq. 2,
//            with Z symmetric so Z_ts = Z(s, t)^T).
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <thread>

#include "h2_host.h"

namespace h2 {
namespace {

struct KernelCtx {
  const double* pts;  // global order
  const double* sq;   // sqrt(chi), global order
  const double* chi;
  double k, sign, self_re, self_im, w;  // w = k^2 h^3 / (4 pi)
};

inline cplx zentry(const KernelCtx& K, int64_t i, int64_t j) {
  if (i == j) return cplx(1.0 + K.sign * K.chi[i] * K.self_re, K.sign * K.chi[i] * K.self_im);
  const double dx = K.pts[3 * i] - K.pts[3 * j], dy = K.pts[3 * i + 1] - K.pts[3 * j + 1],
               dz = K.pts[3 * i + 2] - K.pts[3 * j + 2];
  const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
  const double a = K.sign * K.sq[i] * K.sq[j] * K.w / r;
  return cplx(a * std::cos(K.k * r), -a * std::sin(K.k * r));
}

// column-major helpers
struct Mat {
  int m = 0, n = 0;
  std::vector<cplx> a;
  Mat() = default;
  Mat(int m_, int n_) : m(m_), n(n_), a((size_t)m_ * n_) {}
  cplx& operator()(int i, int j) { return a[(size_t)i + (size_t)j * m]; }
  const cplx& operator()(int i, int j) const { return a[(size_t)i + (size_t)j * m]; }
};

// Householder vector for x (len n): returns tau, overwrites x with v (v0 = 1),
// beta in *beta.  H = I - tau v v^H, H^H x = beta e1.
cplx householder(cplx* x, int n, double* beta) {
  double s = 0;
  for (int i = 1; i < n; ++i) s += std::norm(x[i]);
  const cplx al = x[0];
  if (s == 0.0 && al.imag() == 0.0) {
    *beta = al.real();
    x[0] = 1.0;
    return 0.0;
  }
  const double nrm = std::sqrt(std::norm(al) + s);
  const double b = al.real() >= 0 ? -nrm : nrm;
  const cplx tau((b - al.real()) / b, -al.imag() / b);
  const cplx sc = 1.0 / (al - b);
  for (int i = 1; i < n; ++i) x[i] *= sc;
  x[0] = 1.0;
  *beta = b;
  return tau;
}

// Row interpolative decomposition from the Gram G = M M^H (nr x nr):
// skeleton rows and P (nr x k) with M ~= P M(skel, :).
void row_id_gram(const Mat& G, double eps, std::vector<int>& skel, Mat& P) {
  const int nr = G.m;
  std::vector<double> d(nr);
  for (int i = 0; i < nr; ++i) d[i] = G(i, i).real();
  std::vector<int> piv(nr);
  for (int i = 0; i < nr; ++i) piv[i] = i;
  Mat Lm(nr, nr);  // row = original index, column = step
  double first = -1;
  int k = 0;
  for (int j = 0; j < nr; ++j) {
    int best = j;
    for (int i = j + 1; i < nr; ++i)
      if (d[piv[i]] > d[piv[best]]) best = i;
    const double dv = d[piv[best]];
    if (j == 0) first = dv;
    if (!(dv > eps * eps * first) || dv <= 0.0) break;
    std::swap(piv[j], piv[best]);
    const int p = piv[j];
    const double sd = std::sqrt(dv);
    for (int q = j; q < nr; ++q) {
      const int i = piv[q];
      cplx v = G(i, p);
      for (int t = 0; t < j; ++t) v -= Lm(i, t) * std::conj(Lm(p, t));
      Lm(i, j) = v / sd;
    }
    for (int q = j + 1; q < nr; ++q) d[piv[q]] -= std::norm(Lm(piv[q], j));
    k = j + 1;
  }
  skel.assign(piv.begin(), piv.begin() + k);
  P = Mat(nr, k);
  for (int j = 0; j < k; ++j) P(piv[j], j) = 1.0;
  // other rows: x L_s = L_r(i, :) with L_s = L(skel, :) lower triangular
  std::vector<cplx> x(k);
  for (int q = k; q < nr; ++q) {
    const int i = piv[q];
    for (int j = k - 1; j >= 0; --j) {
      cplx v = Lm(i, j);
      for (int t = j + 1; t < k; ++t) v -= x[t] * Lm(piv[t], j);
      x[j] = v / Lm(piv[j], j);
    }
    for (int j = 0; j < k; ++j) P(i, j) = x[j];
  }
}

// thin QR by Householder: P (m x k) = Q R, Q orthonormal (m x k), R (k x k)
void thin_qr(const Mat& P, Mat& Q, Mat& R) {
  const int m = P.m, k = P.n;
  Mat A = P;
  std::vector<cplx> tau(k);
  R = Mat(k, k);
  for (int j = 0; j < k; ++j) {
    double beta;
    tau[j] = householder(&A(j, j), m - j, &beta);
    for (int c = j + 1; c < k; ++c) {
      cplx d = 0;
      for (int i = j; i < m; ++i) d += std::conj(A(i, j)) * A(i, c);
      d *= std::conj(tau[j]);
      for (int i = j; i < m; ++i) A(i, c) -= A(i, j) * d;
    }
    R(j, j) = beta;
    for (int c = j + 1; c < k; ++c) R(j, c) = A(j, c);
  }
  Q = Mat(m, k);
  for (int j = 0; j < k; ++j) Q(j, j) = 1.0;
  for (int j = k - 1; j >= 0; --j) {
    for (int c = 0; c < k; ++c) {
      cplx d = Q(j, c);
      for (int i = j + 1; i < m; ++i) d += std::conj(A(i, j)) * Q(i, c);
      d *= tau[j];
      Q(j, c) -= d;
      for (int i = j + 1; i < m; ++i) Q(i, c) -= A(i, j) * d;
    }
  }
}

template <class F>
void parallel_for(int n, F f) {
  const int nt = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto& x : th) x.join();
}

}  // namespace

// Orthonormal complement of the orthonormal columns of B (n x k): the last
// n - k columns of the Householder Q of B (Step 1, eq. 4, computed once when
// the H^2 matrix is set up: the paper notes V^perp may be stored then).
std::vector<cplx> host_complement(const std::vector<cplx>& B, int n, int k) {
  Mat A(n, k);
  A.a = B;
  std::vector<cplx> tau(k);
  for (int j = 0; j < k; ++j) {
    double beta;
    tau[j] = householder(&A(j, j), n - j, &beta);
    for (int c = j + 1; c < k; ++c) {
      cplx d = 0;
      for (int i = j; i < n; ++i) d += std::conj(A(i, j)) * A(i, c);
      d *= std::conj(tau[j]);
      for (int i = j; i < n; ++i) A(i, c) -= A(i, j) * d;
    }
  }
  const int q = n - k;
  Mat E(n, q);
  for (int c = 0; c < q; ++c) E(k + c, c) = 1.0;
  for (int j = k - 1; j >= 0; --j)
    for (int c = 0; c < q; ++c) {
      cplx d = E(j, c);
      for (int i = j + 1; i < n; ++i) d += std::conj(A(i, j)) * E(i, c);
      d *= tau[j];
      E(j, c) -= d;
      for (int i = j + 1; i < n; ++i) E(i, c) -= A(i, j) * d;
    }
  return E.a;
}

void host_gram(const double* pts, const double* sq, double k, double w, const std::vector<std::vector<int64_t>>& rows,
               const std::vector<std::vector<int64_t>>& ranges, std::vector<std::vector<cplx>>& G) {
  G.assign(rows.size(), {});
  parallel_for((int)rows.size(), [&](int t) {
    const int nr = (int)rows[t].size();
    std::vector<cplx> g((size_t)nr * nr, 0.0), z(nr);
    for (size_t q = 0; q + 1 < ranges[t].size(); q += 2)
      for (int64_t c = ranges[t][q]; c < ranges[t][q] + ranges[t][q + 1]; ++c) {
        for (int i = 0; i < nr; ++i) {
          const int64_t p = rows[t][i];
          const double dx = pts[3 * p] - pts[3 * c], dy = pts[3 * p + 1] - pts[3 * c + 1],
                       dz = pts[3 * p + 2] - pts[3 * c + 2];
          const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
          const double a = w * sq[p] * sq[c] / r;
          z[i] = cplx(a * std::cos(k * r), -a * std::sin(k * r));
        }
        for (int j = 0; j < nr; ++j) {
          const cplx zj = std::conj(z[j]);
          for (int i = 0; i < nr; ++i) g[(size_t)i + (size_t)j * nr] += z[i] * zj;
        }
      }
    G[t] = std::move(g);
  });
}

std::string build_h2(const double* pts, int64_t N, double k, double h, const double* chi, int64_t chi_len,
                     double eps, const h2_opts& o, H2Host& H, const GramFn& gram) {
  std::vector<double> chiv(N), sq(N);
  for (int64_t i = 0; i < N; ++i) {
    chiv[i] = chi_len == 1 ? chi[0] : chi[i];
    if (!(chiv[i] > 0)) return "chi must be > 0 for every cell";
    sq[i] = std::sqrt(chiv[i]);
  }
  build_tree(pts, N, o.leafsize, H.tree);
  build_partition(H.tree, o.eta, H.part);
  const Tree& T = H.tree;
  const Partition& Pt = H.part;
  const int L = T.L, l0 = Pt.l0;
  H.L = L;
  H.l0 = l0;
  H.dscale = sq;
  const double a = std::cbrt(3.0 / (4.0 * M_PI)) * h;
  const cplx self = (1.0 + cplx(0, k * a)) * std::exp(cplx(0, -k * a)) - 1.0;
  KernelCtx K{pts, sq.data(), chiv.data(), k, o.sign, self.real(), self.imag(), k * k * h * h * h / (4.0 * M_PI)};

  std::vector<std::vector<std::vector<int>>> admp(L + 1);
  for (int l = 0; l <= L; ++l) {
    admp[l].assign(size_t(1) << l, {});
    for (auto [t, s] : Pt.adm[l]) admp[l][t].push_back(s);
  }
  // proxy construction (h2_opts.proxy_min > 0): the far field F*(t) of a
  // cluster is sampled by the points of F*(t) inside the sphere of radius
  // R = proxy_radius * r_t around c_t plus proxy points on two concentric
  // spheres (radii R and 0.8 R, both enclosing t) that stand for the sources
  // outside R; per sphere max(proxy_min, ceil(2 (k R + 10)^2)) Fibonacci
  // points, weighted so that their sample matches the far field's strength
  // sum_s n_s chi / |c_t - c_s|^2.  O(N k^2) in all instead of O(N^2).
  const bool proxy = o.proxy_min > 0;
  double chimean = 0;
  for (int64_t i = 0; i < N; ++i) chimean += chiv[i];
  chimean /= (double)N;
  std::vector<std::vector<int64_t>> proxy_off(L + 1);  // first proxy position of each cluster
  std::vector<std::vector<int>> proxy_cnt(L + 1);
  if (proxy) {
    H.proxy_pts.clear();
    H.proxy_w.clear();
    for (int l = l0; l <= L; ++l) {
      proxy_off[l].assign(size_t(1) << l, 0);
      proxy_cnt[l].assign(size_t(1) << l, 0);
      for (int t = 0; t < (1 << l); ++t) {
        // far-field strength estimate from the admissible partners of t and its ancestors
        double far = 0;
        for (int lv = l, anc = t; lv >= 0; --lv, anc >>= 1)
          for (int s : admp[lv][anc]) {
            double d2 = 0;
            for (int q = 0; q < 3; ++q) {
              const double v = T.centre[l][3 * t + q] - T.centre[lv][3 * s + q];
              d2 += v * v;
            }
            far += (double)T.size[lv][s] * chimean / std::max(d2, 1e-300);
          }
        if (far == 0) continue;  // no far field: rank 0
        const double R = o.proxy_radius * T.radius[l][t];
        // the far-field nodes with points outside the sphere: descend the
        // partners' subtrees until a node is wholly inside (sampled exactly,
        // point by point) or wholly outside, or is a leaf with points on both
        // sides; their directions and angular radii seen from c_t decide
        // which proxy points are placed (a proxy stands for the outside
        // sources near its direction); none at all when every far point is
        // inside
        std::vector<std::array<double, 4>> cones;  // unit direction, angular radius
        {
          std::vector<std::pair<int, int>> st;
          for (int lv = l, anc = t; lv >= 0; --lv, anc >>= 1)
            for (int s : admp[lv][anc]) st.push_back({lv, s});
          while (!st.empty()) {
            const auto [ll, u] = st.back();
            st.pop_back();
            double dv[3], d2 = 0;
            for (int q = 0; q < 3; ++q) {
              dv[q] = T.centre[ll][3 * u + q] - T.centre[l][3 * t + q];
              d2 += dv[q] * dv[q];
            }
            const double d = std::sqrt(d2), ru = T.radius[ll][u];
            if (d + ru <= R) continue;  // wholly inside
            bool rec = d - ru > R;      // wholly outside
            if (!rec && ll == L) {
              for (int64_t p = T.start[L][u]; p < T.start[L][u] + T.size[L][u] && !rec; ++p) {
                double e2 = 0;
                for (int q = 0; q < 3; ++q) {
                  const double v = T.centre[l][3 * t + q] - pts[3 * T.perm[p] + q];
                  e2 += v * v;
                }
                rec = e2 > R * R;
              }
              if (!rec) continue;
            }
            if (rec) {
              const double ang = d > ru ? std::asin(std::min(1.0, ru / d)) : M_PI;
              cones.push_back({dv[0] / d, dv[1] / d, dv[2] / d, ang});
            } else {
              st.push_back({ll + 1, 2 * u});
              st.push_back({ll + 1, 2 * u + 1});
            }
          }
        }
        proxy_cnt[l][t] = -1;  // far field present (sampled inside R only)
        if (cones.empty()) continue;
        const int np = std::max(o.proxy_min, (int)std::ceil(2.0 * (k * R + 10.0) * (k * R + 10.0)));
        proxy_off[l][t] = N + (int64_t)H.proxy_w.size();
        // weight: sum over the 2 np proxies of w^2 / R_p^2 equals `far`
        const double wgt = std::sqrt(far / (np / (R * R) + np / (0.64 * R * R)));
        int kept = 0;
        for (int sph = 0; sph < 2; ++sph) {
          const double rad = sph == 0 ? R : 0.8 * R;
          for (int i = 0; i < np; ++i) {
            const double z = 1.0 - 2.0 * (i + 0.5) / np, rr = std::sqrt(std::max(0.0, 1.0 - z * z));
            const double th = M_PI * (1.0 + std::sqrt(5.0)) * (i + 0.5);
            const double u[3] = {rr * std::cos(th), rr * std::sin(th), z};
            bool use = false;
            for (const auto& cn : cones) {
              const double cosa = u[0] * cn[0] + u[1] * cn[1] + u[2] * cn[2];
              if (std::acos(std::max(-1.0, std::min(1.0, cosa))) <= cn[3] + o.proxy_margin) {
                use = true;
                break;
              }
            }
            if (!use) continue;
            H.proxy_pts.push_back(T.centre[l][3 * t] + rad * u[0]);
            H.proxy_pts.push_back(T.centre[l][3 * t + 1] + rad * u[1]);
            H.proxy_pts.push_back(T.centre[l][3 * t + 2] + rad * u[2]);
            H.proxy_w.push_back(wgt);
            ++kept;
          }
        }
        proxy_cnt[l][t] = kept > 0 ? kept : -1;
        if (kept == 0) continue;
      }
    }
  }
  // far-field tree positions of t inside the sphere (c_t, R): descend the
  // admissible partners' subtrees, pruning by bounding spheres
  auto inside_runs = [&](int l, int t, std::vector<int64_t>& out) {
    const double R = o.proxy_radius * T.radius[l][t];
    const double* ct = &T.centre[l][3 * t];
    std::vector<int64_t> pos;
    std::vector<std::pair<int, int>> stack;
    for (int lv = l, anc = t; lv >= 0; --lv, anc >>= 1)
      for (int s : admp[lv][anc]) stack.push_back({lv, s});
    while (!stack.empty()) {
      const auto [ll, u] = stack.back();
      stack.pop_back();
      double d2 = 0;
      for (int q = 0; q < 3; ++q) {
        const double v = ct[q] - T.centre[ll][3 * u + q];
        d2 += v * v;
      }
      if (std::sqrt(d2) - T.radius[ll][u] > R) continue;
      if (ll == L) {
        for (int64_t p = T.start[L][u]; p < T.start[L][u] + T.size[L][u]; ++p) {
          const int64_t g = T.perm[p];
          double e2 = 0;
          for (int q = 0; q < 3; ++q) {
            const double v = ct[q] - pts[3 * g + q];
            e2 += v * v;
          }
          if (e2 <= R * R) pos.push_back(p);
        }
      } else {
        stack.push_back({ll + 1, 2 * u});
        stack.push_back({ll + 1, 2 * u + 1});
      }
    }
    std::sort(pos.begin(), pos.end());
    for (size_t i = 0; i < pos.size();) {
      size_t j = i + 1;
      while (j < pos.size() && pos[j] == pos[j - 1] + 1) ++j;
      out.push_back(pos[i]);
      out.push_back((int64_t)(j - i));
      i = j;
    }
  };
  H.rank.assign(L + 1, {});
  H.V.assign(size_t(1) << L, {});
  H.T.assign(L + 1, {});
  H.S.assign(L + 1, {});
  std::vector<std::vector<std::vector<int64_t>>> skel(L + 1);  // tree positions
  std::vector<std::vector<Mat>> Rm(L + 1);

  for (int l = L; l >= l0; --l) {
    const int nc = 1 << l;
    skel[l].assign(nc, {});
    Rm[l].assign(nc, Mat());
    H.rank[l].assign(nc, 0);
    if (l < L) H.T[l].assign(nc, {});
    std::vector<std::vector<int64_t>> rows(nc), ranges(nc);
    for (int t = 0; t < nc; ++t) {
      if (l == L) {
        for (int64_t p = T.start[l][t]; p < T.start[l][t] + T.size[l][t]; ++p) rows[t].push_back(p);
      } else {
        rows[t] = skel[l + 1][2 * t];
        rows[t].insert(rows[t].end(), skel[l + 1][2 * t + 1].begin(), skel[l + 1][2 * t + 1].end());
      }
      if (proxy) {
        if (proxy_cnt[l][t] > 0) {
          ranges[t].push_back(proxy_off[l][t]);
          ranges[t].push_back(proxy_cnt[l][t]);
        }
        if (proxy_cnt[l][t] != 0) inside_runs(l, t, ranges[t]);
      } else {
        for (int lv = l, anc = t; lv >= 0; --lv, anc >>= 1)
          for (int s : admp[lv][anc]) {
            ranges[t].push_back(T.start[lv][s]);
            ranges[t].push_back(T.size[lv][s]);
          }
      }
      if (ranges[t].empty()) rows[t].clear();  // no far field: rank 0
    }
    std::vector<std::vector<cplx>> G;
    auto tg = std::chrono::steady_clock::now();
    gram(l, rows, ranges, G);
    H.t_gram_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tg).count();
    tg = std::chrono::steady_clock::now();
    parallel_for(nc, [&](int t) {
      const int nr = (int)rows[t].size();
      std::vector<int> sk;
      Mat P(nr, 0);
      if (nr > 0) {
        Mat Gm(nr, nr);
        Gm.a = G[t];
        row_id_gram(Gm, eps, sk, P);
      }
      const int kk = (int)sk.size();
      std::vector<int64_t> sg(kk);
      for (int j = 0; j < kk; ++j) sg[j] = rows[t][sk[j]];
      skel[l][t] = sg;
      H.rank[l][t] = kk;
      Mat Q, R;
      if (l == L) {
        thin_qr(P, Q, R);
        H.V[t] = Q.a;
      } else {
        const Mat& R1 = Rm[l + 1][2 * t];
        const Mat& R2 = Rm[l + 1][2 * t + 1];
        const int k1 = R1.m, k2 = R2.m;
        Mat Pm(k1 + k2, kk);
        if (nr > 0)
          for (int j = 0; j < kk; ++j) {
            for (int i = 0; i < k1; ++i) {
              cplx v = 0;
              for (int q = i; q < k1; ++q) v += R1(i, q) * P(q, j);
              Pm(i, j) = v;
            }
            for (int i = 0; i < k2; ++i) {
              cplx v = 0;
              for (int q = i; q < k2; ++q) v += R2(i, q) * P(k1 + q, j);
              Pm(k1 + i, j) = v;
            }
          }
        thin_qr(Pm, Q, R);
        H.T[l][t] = Q.a;
      }
      Rm[l][t] = R;
    });
    H.t_id_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tg).count();
  }
  // couplings of admissible pairs, levels l0..L
  auto tc = std::chrono::steady_clock::now();
  for (int l = l0; l <= L; ++l) {
    const auto& pairs = Pt.adm[l];
    H.S[l].assign(pairs.size(), {});
    parallel_for((int)pairs.size(), [&](int q) {
      const int t = pairs[q].first, s = pairs[q].second;
      const auto& st = skel[l][t];
      const auto& ss = skel[l][s];
      const int kt = (int)st.size(), ks = (int)ss.size();
      Mat Zs(kt, ks);
      for (int j = 0; j < ks; ++j)
        for (int i = 0; i < kt; ++i) Zs(i, j) = zentry(K, T.perm[st[i]], T.perm[ss[j]]);
      const Mat& Rt = Rm[l][t];
      const Mat& Rs = Rm[l][s];
      Mat Y(kt, ks);  // Rt Zs
      for (int j = 0; j < ks; ++j)
        for (int i = 0; i < kt; ++i) {
          cplx v = 0;
          for (int p = i; p < kt; ++p) v += Rt(i, p) * Zs(p, j);
          Y(i, j) = v;
        }
      Mat Sm(kt, ks);  // Y Rs^T
      for (int j = 0; j < ks; ++j)
        for (int i = 0; i < kt; ++i) {
          cplx v = 0;
          for (int p = j; p < ks; ++p) v += Y(i, p) * Rs(j, p);
          Sm(i, j) = v;
        }
      H.S[l][q] = Sm.a;
    });
  }
  H.t_coupling_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc).count();
  tc = std::chrono::steady_clock::now();
  // dense near-field blocks at the leaf level
  const auto& np_ = Pt.inad[L];
  H.D.assign(np_.size(), {});
  parallel_for((int)np_.size(), [&](int q) {
    const int t = np_[q].first, s = np_[q].second;
    const int64_t at = T.start[L][t], as = T.start[L][s];
    const int nt = (int)T.size[L][t], ns = (int)T.size[L][s];
    std::vector<cplx> Dm((size_t)nt * ns);
    for (int j = 0; j < ns; ++j)
      for (int i = 0; i < nt; ++i) Dm[(size_t)i + (size_t)j * nt] = zentry(K, T.perm[at + i], T.perm[as + j]);
    H.D[q] = std::move(Dm);
  });
  H.t_near_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc).count();
  return "";
}

// New contrast on an existing representation: Z' = I + E (Z - I) E with
// E = diag(e) (tree order), e_i = sqrt(chi'_i / chi_i).  Exact algebra on the
// H^2 form (no new approximation, ranks unchanged): dense near blocks are
// scaled entrywise; the scaled bases E_t V_t are re-orthonormalised from the
// leaves up, E_t V_t = Q_t R_t (leaf: V'_t = Q_t; parent:
// diag(R_t1, R_t2) T_t = Q_t R_t, T'_t = Q_t), which keeps them nested
// (eq. 3); couplings become S'_ts = R_t S_ts R_s^T (eq. 2).
void rescale_h2(H2Host& H, const std::vector<double>& e) {
  const Tree& T = H.tree;
  const int L = H.L, l0 = H.l0;
  std::vector<std::vector<Mat>> Rm(L + 1);
  for (int l = L; l >= l0; --l) {
    const int nc = 1 << l;
    Rm[l].assign(nc, Mat());
    parallel_for(nc, [&](int t) {
      const int k = H.rank[l][t];
      Mat A;
      if (l == L) {
        const int n = (int)T.size[L][t];
        A = Mat(n, k);
        A.a = H.V[t];
        for (int j = 0; j < k; ++j)
          for (int i = 0; i < n; ++i) A(i, j) *= e[T.start[L][t] + i];
      } else {
        const Mat& R1 = Rm[l + 1][2 * t];
        const Mat& R2 = Rm[l + 1][2 * t + 1];
        const int k1 = R1.m, k2 = R2.m;
        Mat Tm(k1 + k2, k);
        Tm.a = H.T[l][t];
        A = Mat(k1 + k2, k);
        for (int j = 0; j < k; ++j) {
          for (int i = 0; i < k1; ++i) {
            cplx v = 0;
            for (int q = i; q < k1; ++q) v += R1(i, q) * Tm(q, j);
            A(i, j) = v;
          }
          for (int i = 0; i < k2; ++i) {
            cplx v = 0;
            for (int q = i; q < k2; ++q) v += R2(i, q) * Tm(k1 + q, j);
            A(k1 + i, j) = v;
          }
        }
      }
      Mat Q, R;
      thin_qr(A, Q, R);
      if (l == L) H.V[t] = Q.a;
      else H.T[l][t] = Q.a;
      Rm[l][t] = R;
    });
  }
  for (int l = l0; l <= L; ++l) {
    const auto& pairs = H.part.adm[l];
    parallel_for((int)pairs.size(), [&](int q) {
      const int t = pairs[q].first, s = pairs[q].second;
      const Mat& Rt = Rm[l][t];
      const Mat& Rs = Rm[l][s];
      const int kt = Rt.m, ks = Rs.m;
      Mat S(kt, ks);
      S.a = H.S[l][q];
      Mat Y(kt, ks);  // Rt S
      for (int j = 0; j < ks; ++j)
        for (int i = 0; i < kt; ++i) {
          cplx v = 0;
          for (int p = i; p < kt; ++p) v += Rt(i, p) * S(p, j);
          Y(i, j) = v;
        }
      for (int j = 0; j < ks; ++j)  // Y Rs^T
        for (int i = 0; i < kt; ++i) {
          cplx v = 0;
          for (int p = j; p < ks; ++p) v += Y(i, p) * Rs(j, p);
          S(i, j) = v;
        }
      H.S[l][q] = S.a;
    });
  }
  const auto& np_ = H.part.inad[L];
  parallel_for((int)np_.size(), [&](int q) {
    const int t = np_[q].first, s = np_[q].second;
    const int64_t at = T.start[L][t], as = T.start[L][s];
    const int nt = (int)T.size[L][t], ns = (int)T.size[L][s];
    std::vector<cplx>& D = H.D[q];
    for (int j = 0; j < ns; ++j)
      for (int i = 0; i < nt; ++i) {
        const double f = e[at + i] * e[as + j];
        cplx& z = D[(size_t)i + (size_t)j * nt];
        z = (t == s && i == j) ? 1.0 + f * (z - 1.0) : f * z;
      }
  });
}

}  // namespace h2
