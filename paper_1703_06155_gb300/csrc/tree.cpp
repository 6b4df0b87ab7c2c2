// Cluster tree and block partition (Sec. II, eq. 1), host side.
//
//  * bisection along the longest axis of the cluster's bounding box (ties ->
//    lowest axis), points ordered by (coordinate, global index), the first
//    ceil(n/2) go to the left child;
//  * all clusters split to one depth L = min{L : ceil(N/2^L) <= leafsize}, so
//    level l has exactly 2^l clusters;
//  * (t, s) admissible iff t != s and ||c_t - c_s|| >= eta (r_t + r_s),
//    c = bounding-box centre, r = largest distance from c to a point of the
//    cluster.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "h2_host.h"

namespace h2 {

void build_tree(const double* pts, int64_t N, int leafsize, Tree& t) {
  t.N = N;
  int L = 0;
  while ((N + (int64_t(1) << L) - 1) / (int64_t(1) << L) > leafsize) ++L;
  t.L = L;
  t.perm.resize(N);
  std::iota(t.perm.begin(), t.perm.end(), 0);
  t.start.assign(L + 1, {});
  t.size.assign(L + 1, {});
  t.start[0] = {0};
  t.size[0] = {N};
  std::vector<std::pair<double, int64_t>> key;
  for (int l = 0; l < L; ++l) {
    for (size_t c = 0; c < t.start[l].size(); ++c) {
      const int64_t s = t.start[l][c], n = t.size[l][c];
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int64_t p = s; p < s + n; ++p)
        for (int d = 0; d < 3; ++d) {
          const double v = pts[3 * t.perm[p] + d];
          lo[d] = std::min(lo[d], v);
          hi[d] = std::max(hi[d], v);
        }
      int ax = 0;
      for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
      key.resize(n);
      for (int64_t p = 0; p < n; ++p) key[p] = {pts[3 * t.perm[s + p] + ax], t.perm[s + p]};
      std::sort(key.begin(), key.end());
      for (int64_t p = 0; p < n; ++p) t.perm[s + p] = key[p].second;
      const int64_t n1 = (n + 1) / 2;
      t.start[l + 1].push_back(s);
      t.size[l + 1].push_back(n1);
      t.start[l + 1].push_back(s + n1);
      t.size[l + 1].push_back(n - n1);
    }
  }
  t.centre.assign(L + 1, {});
  t.radius.assign(L + 1, {});
  for (int l = 0; l <= L; ++l) {
    for (size_t c = 0; c < t.start[l].size(); ++c) {
      const int64_t s = t.start[l][c], n = t.size[l][c];
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int64_t p = s; p < s + n; ++p)
        for (int d = 0; d < 3; ++d) {
          const double v = pts[3 * t.perm[p] + d];
          lo[d] = std::min(lo[d], v);
          hi[d] = std::max(hi[d], v);
        }
      double cc[3];
      for (int d = 0; d < 3; ++d) cc[d] = 0.5 * (lo[d] + hi[d]);
      double r2 = 0;
      for (int64_t p = s; p < s + n; ++p) {
        double q = 0;
        for (int d = 0; d < 3; ++d) {
          const double v = pts[3 * t.perm[p] + d] - cc[d];
          q += v * v;
        }
        r2 = std::max(r2, q);
      }
      for (int d = 0; d < 3; ++d) t.centre[l].push_back(cc[d]);
      t.radius[l].push_back(std::sqrt(r2));
    }
  }
}

void build_partition(const Tree& t, double eta, Partition& p) {
  const int L = t.L;
  p.adm.assign(L + 1, {});
  p.inad.assign(L + 1, {});
  std::vector<Pair> cur{{0, 0}}, nxt;
  for (int l = 0; l <= L; ++l) {
    nxt.clear();
    for (auto [a, b] : cur) {
      double d2 = 0;
      for (int q = 0; q < 3; ++q) {
        const double v = t.centre[l][3 * a + q] - t.centre[l][3 * b + q];
        d2 += v * v;
      }
      // a cluster is never admissible with itself (eq. (1) holds for it only
      // when its diameter is zero, and its block holds the singular self term)
      if (a != b && std::sqrt(d2) >= eta * (t.radius[l][a] + t.radius[l][b])) {
        p.adm[l].push_back({a, b});
      } else {
        p.inad[l].push_back({a, b});
        if (l < L)
          for (int x = 2 * a; x <= 2 * a + 1; ++x)
            for (int y = 2 * b; y <= 2 * b + 1; ++y) nxt.push_back({x, y});
      }
    }
    std::sort(p.adm[l].begin(), p.adm[l].end());
    std::sort(p.inad[l].begin(), p.inad[l].end());
    cur.swap(nxt);
  }
  p.l0 = L;
  for (int l = L; l >= 0; --l)
    if (!p.adm[l].empty()) p.l0 = l;
}

std::vector<std::vector<int>> near_lists(const Partition& p, int l) {
  std::vector<std::vector<int>> nb(size_t(1) << l);
  for (auto [a, b] : p.inad[l]) nb[a].push_back(b);
  for (auto& v : nb) std::sort(v.begin(), v.end());
  return nb;
}

// Smallest colour not used by an already coloured near neighbour, visiting
// clusters in increasing index; a colour class has no two near neighbours.
// Colouring of the near-field graph by saturation degree: repeatedly colour
// the uncoloured cluster with the most distinct neighbour colours (ties: more
// neighbours, then the lowest index) with the smallest colour its neighbours
// do not use.  Clusters of one colour are never near neighbours.
std::vector<int> greedy_colours(const std::vector<std::vector<int>>& nbrs) {
  const int n = (int)nbrs.size();
  std::vector<int> col(n, -1), deg(n, 0), nsat(n, 0);
  std::vector<std::vector<char>> seen(n);  // seen[i][c]: colour c among i's neighbours
  for (int i = 0; i < n; ++i)
    for (int j : nbrs[i])
      if (j != i) ++deg[i];
  std::vector<char> used;
  for (int step = 0; step < n; ++step) {
    int bi = -1;
    for (int i = 0; i < n; ++i) {
      if (col[i] >= 0) continue;
      if (bi < 0 || nsat[i] > nsat[bi] || (nsat[i] == nsat[bi] && deg[i] > deg[bi])) bi = i;
    }
    used.assign(n + 1, 0);
    for (int j : nbrs[bi])
      if (j != bi && col[j] >= 0) used[col[j]] = 1;
    int c = 0;
    while (used[c]) ++c;
    col[bi] = c;
    for (int j : nbrs[bi]) {
      if (j == bi || col[j] >= 0) continue;
      if ((int)seen[j].size() <= c) seen[j].resize(c + 1, 0);
      if (!seen[j][c]) {
        seen[j][c] = 1;
        ++nsat[j];
      }
    }
  }
  return col;
}

}  // namespace h2
