// h2_build: H^2 representation of Z = I + s D^{1/2} K D^{1/2} by proxy
// sampling and nested interpolative decompositions (host, multi-threaded).
//
// The paper builds its H^2 matrices with the method of its refs. [14], [15]
// and does not describe it (Sec. VI).  This construction, for each level from
// the leaves up and each cluster t:
//   rows_t   the points of t (leaf) or the skeletons of its two children
//   sample   Z(rows_t, cols) with cols = every point of t's far field
//            (clusters admissible with t or an ancestor of t) inside a sphere
//            of radius proxy_radius * r_t around c_t, plus, if some far point
//            lies outside it, single- and double-layer sources on that sphere
//            (Fibonacci points): by Green's representation formula they span
//            the field of every far source outside the sphere.
//   ID       column-pivoted Householder QR of sample^T, stopped when the
//            largest remaining column norm <= eps * the first one; the pivots
//            are the skeleton rows, P_t interpolates the other rows.
//   basis    P_t = Q R (leaf: V_t = Q) or diag(R_t1, R_t2) P_t = Q R
//            (non-leaf: T_t = Q), so the bases are orthonormal and nested
//            (eq. 3); couplings S_ts = R_t Z(skel_t, skel_s) R_s^T (eq. 2,
//            with Z symmetric so Z_ts = Z(s, t)^T).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include "h2_host.h"

namespace h2 {
namespace {

struct KernelCtx {
  const double* pts;
  const double* sq;   // sqrt(chi), global index
  const double* chi;
  double k, h, sign, self_re, self_im, w;  // w = k^2 h^3 / (4 pi)
};

inline cplx zentry(const KernelCtx& K, int64_t i, int64_t j) {
  if (i == j) return cplx(1.0 + K.sign * K.chi[i] * K.self_re, K.sign * K.chi[i] * K.self_im);
  const double dx = K.pts[3 * i] - K.pts[3 * j], dy = K.pts[3 * i + 1] - K.pts[3 * j + 1],
               dz = K.pts[3 * i + 2] - K.pts[3 * j + 2];
  const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
  const double a = K.sign * K.sq[i] * K.sq[j] * K.w / r;
  return cplx(a * std::cos(K.k * r), -a * std::sin(K.k * r));
}

// Green's function G = e^{-jkr}/(4 pi r) scaled by k^2 h^3 (single layer) and
// its derivative along the outward sphere normal at the source (double layer)
inline void proxy_entry(const KernelCtx& K, int64_t i, const double* z, const double* nz, cplx& g, cplx& dg) {
  const double dx = K.pts[3 * i] - z[0], dy = K.pts[3 * i + 1] - z[1], dz = K.pts[3 * i + 2] - z[2];
  const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
  const cplx e = std::exp(cplx(0, -K.k * r));
  g = K.sq[i] * K.w * e / r;
  // d/dn_z of e^{-jkr}/r with r = |x - z|: (jk r + 1) e^{-jkr} / r^2 * ((x-z).n / r)
  const double cosn = (dx * nz[0] + dy * nz[1] + dz * nz[2]) / r;
  dg = K.sq[i] * K.w * cplx(1.0, K.k * r) * e / (r * r) * cosn;
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

// Row interpolative decomposition of M (nr x nc): skeleton rows and P (nr x k)
// with M ~= P M(skel, :).
void row_id(const Mat& M, double eps, std::vector<int>& skel, Mat& P) {
  const int nr = M.m, nc = M.n;
  // A = M^T (nc x nr), pivot over its columns (= rows of M)
  Mat A(nc, nr);
  for (int j = 0; j < nr; ++j)
    for (int i = 0; i < nc; ++i) A(i, j) = M(j, i);
  std::vector<int> piv(nr);
  for (int j = 0; j < nr; ++j) piv[j] = j;
  std::vector<double> cn(nr);
  const int kmax = std::min(nr, nc);
  double first = -1;
  int k = 0;
  for (int j = 0; j < kmax; ++j) {
    int best = j;
    double bv = -1;
    for (int c = j; c < nr; ++c) {
      double s = 0;
      for (int i = j; i < nc; ++i) s += std::norm(A(i, c));
      cn[c] = s;
      if (s > bv) { bv = s; best = c; }
    }
    const double bn = std::sqrt(bv);
    if (j == 0) first = bn;
    if (bn <= eps * first || bn == 0.0) break;
    if (best != j) {
      for (int i = 0; i < nc; ++i) std::swap(A(i, j), A(i, best));
      std::swap(piv[j], piv[best]);
    }
    double beta;
    const cplx tau = householder(&A(j, j), nc - j, &beta);
    // apply H^H = I - conj(tau) v v^H to A(j:, j+1:)
    for (int c = j + 1; c < nr; ++c) {
      cplx d = 0;
      for (int i = j; i < nc; ++i) d += std::conj(A(i, j)) * A(i, c);
      d *= std::conj(tau);
      for (int i = j; i < nc; ++i) A(i, c) -= A(i, j) * d;
    }
    A(j, j) = beta;
    k = j + 1;
  }
  // X = R11^{-1} R12  (k x (nr-k)); R11 upper triangular in A(0:k, 0:k)
  Mat X(k, nr - k);
  for (int c = 0; c < nr - k; ++c) {
    for (int i = k - 1; i >= 0; --i) {
      cplx v = A(i, k + c);
      for (int t = i + 1; t < k; ++t) v -= A(i, t) * X(t, c);
      X(i, c) = v / A(i, i);
    }
  }
  skel.assign(piv.begin(), piv.begin() + k);
  P = Mat(nr, k);
  for (int j = 0; j < k; ++j) P(piv[j], j) = 1.0;
  for (int c = 0; c < nr - k; ++c)
    for (int j = 0; j < k; ++j) P(piv[k + c], j) = X(j, c);
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

std::string build_h2(const double* pts, int64_t N, double k, double h, const double* chi, int64_t chi_len,
                     double eps, const h2_opts& o, H2Host& H) {
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
  KernelCtx K{pts, sq.data(), chiv.data(), k, h, o.sign, self.real(), self.imag(), k * k * h * h * h / (4.0 * M_PI)};

  // admissible partners per level and cluster
  std::vector<std::vector<std::vector<int>>> admp(L + 1);
  for (int l = 0; l <= L; ++l) {
    admp[l].assign(size_t(1) << l, {});
    for (auto [t, s] : Pt.adm[l]) admp[l][t].push_back(s);
  }
  H.rank.assign(L + 1, {});
  H.V.assign(size_t(1) << L, {});
  H.T.assign(L + 1, {});
  H.S.assign(L + 1, {});
  std::vector<std::vector<std::vector<int64_t>>> skel(L + 1);  // global indices
  std::vector<std::vector<Mat>> Rm(L + 1);

  for (int l = L; l >= l0; --l) {
    const int nc = 1 << l;
    skel[l].assign(nc, {});
    Rm[l].assign(nc, Mat());
    H.rank[l].assign(nc, 0);
    if (l < L) H.T[l].assign(nc, {});
    parallel_for(nc, [&](int t) {
      std::vector<int64_t> rows;
      if (l == L) {
        for (int64_t p = T.start[l][t]; p < T.start[l][t] + T.size[l][t]; ++p) rows.push_back(T.perm[p]);
      } else {
        rows = skel[l + 1][2 * t];
        rows.insert(rows.end(), skel[l + 1][2 * t + 1].begin(), skel[l + 1][2 * t + 1].end());
      }
      const double* c = &T.centre[l][3 * t];
      const double rho = o.proxy_radius * T.radius[l][t];
      // far-field points inside the proxy sphere
      std::vector<int64_t> inside;
      bool any_far = false, any_outside = false;
      for (int lv = l, anc = t; lv >= 0; --lv, anc >>= 1) {
        for (int s : admp[lv][anc]) {
          any_far = true;
          const double* cs = &T.centre[lv][3 * s];
          const double dc = std::sqrt((c[0] - cs[0]) * (c[0] - cs[0]) + (c[1] - cs[1]) * (c[1] - cs[1]) +
                                      (c[2] - cs[2]) * (c[2] - cs[2]));
          if (dc >= rho + T.radius[lv][s]) {
            any_outside = true;
            continue;
          }
          for (int64_t p = T.start[lv][s]; p < T.start[lv][s] + T.size[lv][s]; ++p) {
            const int64_t g = T.perm[p];
            double d2 = 0;
            for (int q = 0; q < 3; ++q) d2 += (pts[3 * g + q] - c[q]) * (pts[3 * g + q] - c[q]);
            if (d2 < rho * rho) inside.push_back(g);
            else any_outside = true;
          }
        }
      }
      const int nr = (int)rows.size();
      if (!any_far || nr == 0) {
        skel[l][t].clear();
        Rm[l][t] = Mat(0, 0);
        H.rank[l][t] = 0;
        if (l == L) H.V[t].clear();
        else H.T[l][t].clear();
        return;
      }
      const double kr = k * rho;
      // proxy layers only represent far sources outside the sphere
      int np = (int)std::ceil((kr + 16.0) * (kr + 16.0));
      np = std::max(np, o.proxy_min);
      if (!any_outside) np = 0;
      Mat M(nr, 2 * np + (int)inside.size());
      const double ga = M_PI * (3.0 - std::sqrt(5.0));
      for (int q = 0; q < np; ++q) {
        const double zc = 1.0 - (2.0 * q + 1.0) / np;
        const double rr = std::sqrt(std::max(0.0, 1.0 - zc * zc));
        const double th = ga * q;
        const double nz[3] = {rr * std::cos(th), rr * std::sin(th), zc};
        const double z[3] = {c[0] + rho * nz[0], c[1] + rho * nz[1], c[2] + rho * nz[2]};
        for (int i = 0; i < nr; ++i) {
          cplx g, dg;
          proxy_entry(K, rows[i], z, nz, g, dg);
          M(i, 2 * q) = g;
          M(i, 2 * q + 1) = dg * rho;  // scale the double layer to the single layer
        }
      }
      for (size_t q = 0; q < inside.size(); ++q)
        for (int i = 0; i < nr; ++i) M(i, 2 * np + (int)q) = zentry(K, rows[i], inside[q]);
      std::vector<int> sk;
      Mat P;
      row_id(M, eps, sk, P);
      const int kk = (int)sk.size();
      std::vector<int64_t> sg(kk);
      for (int j = 0; j < kk; ++j) sg[j] = rows[sk[j]];
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
  }
  // couplings of admissible pairs, levels l0..L
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
        for (int i = 0; i < kt; ++i) Zs(i, j) = zentry(K, st[i], ss[j]);
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
  return "";
}

}  // namespace h2
