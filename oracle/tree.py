"""Cluster tree (Sec. II) and block partition by the admissibility test eq. (1).

Readings of what the paper leaves open:
  * bisection of the cluster's points along the longest axis of their bounding
    box (ties -> lowest axis), stable order by (coordinate, global index), the
    left child takes the first ceil(n/2) points;
  * every cluster is split down to one depth L, the smallest with
    ceil(N / 2^L) <= leafsize, so level l holds exactly 2^l clusters as the
    paper's Algorithm 1 assumes;
  * admissibility uses centres and radii: ||c_t - c_s|| >= eta (r_t + r_s)
    for t != s (a cluster is never admissible with itself),
    c = bounding-box centre, r = max distance from c to a point of the cluster.
Clusters at level l are numbered 0..2^l-1; children of c are 2c and 2c+1.
"""
import math

import numpy as np


class ClusterTree:
    def __init__(self, pts, leafsize):
        N = len(pts)
        L = 0
        while math.ceil(N / 2 ** L) > leafsize:
            L += 1
        self.N, self.L, self.leafsize = N, L, leafsize
        perm = np.arange(N)
        starts = [np.array([0])]
        sizes = [np.array([N])]
        for l in range(L):
            ns, nz = [], []
            for s, n in zip(starts[l], sizes[l]):
                idx = perm[s:s + n]
                P = pts[idx]
                ext = P.max(axis=0) - P.min(axis=0)
                axis = int(np.argmax(ext))  # first maximum = lowest axis
                order = np.lexsort((idx, P[:, axis]))
                perm[s:s + n] = idx[order]
                n1 = (n + 1) // 2
                ns += [s, s + n1]
                nz += [n1, n - n1]
            starts.append(np.array(ns))
            sizes.append(np.array(nz))
        self.perm = perm
        self.start = starts
        self.size = sizes
        self.centre, self.radius = [], []
        for l in range(L + 1):
            cs, rs = [], []
            for s, n in zip(starts[l], sizes[l]):
                P = pts[perm[s:s + n]]
                c = 0.5 * (P.max(axis=0) + P.min(axis=0))
                cs.append(c)
                rs.append(float(np.max(np.linalg.norm(P - c, axis=1))))
            self.centre.append(np.array(cs))
            self.radius.append(np.array(rs))

    def indices(self, l, c):
        """Global point indices of cluster c at level l (tree order)."""
        s = self.start[l][c]
        return self.perm[s:s + self.size[l][c]]


class Partition:
    """Admissible / inadmissible block lists per level, by dual traversal.

    Pairs are same-level (t, s); an admissible pair stops the traversal; an
    inadmissible non-leaf pair splits into its 4 child pairs; inadmissible
    leaf pairs are the dense near-field blocks (Sec. II, Fig. 1).
    """

    def __init__(self, tree, eta):
        L = tree.L
        self.adm = [[] for _ in range(L + 1)]
        self.inad = [[] for _ in range(L + 1)]
        cur = [(0, 0)]
        for l in range(L + 1):
            nxt = []
            for t, s in cur:
                d = np.linalg.norm(tree.centre[l][t] - tree.centre[l][s])
                # a cluster is never admissible with itself (eq. (1) holds for
                # it only when its diameter is zero, and its block holds the
                # singular self term)
                if t != s and d >= eta * (tree.radius[l][t] + tree.radius[l][s]):
                    self.adm[l].append((t, s))
                else:
                    self.inad[l].append((t, s))
                    if l < L:
                        for a in (2 * t, 2 * t + 1):
                            for b in (2 * s, 2 * s + 1):
                                nxt.append((a, b))
            self.adm[l].sort()
            self.inad[l].sort()
            cur = nxt
        lv = [l for l in range(L + 1) if self.adm[l]]
        # l0: the minimal level that has admissible blocks (Alg. 1); with no
        # admissible block at all the leaf level is the only level processed.
        self.l0 = min(lv) if lv else L

    def near_lists(self, l):
        """N(i) for every cluster at level l: inadmissible partners incl. i."""
        nb = [[] for _ in range(2 ** l)]
        for t, s in self.inad[l]:
            nb[t].append(s)
        return nb


def greedy_colouring(nbrs):
    """Colouring of the near-field graph by saturation degree (DSatur): repeatedly
    take the uncoloured cluster with the most distinct colours among its
    neighbours (ties: more neighbours, then the lowest index) and give it the
    smallest colour unused by its neighbours.  Clusters of one colour are never
    near neighbours of each other."""
    n = len(nbrs)
    adj = [set(j for j in nbrs[i] if j != i) for i in range(n)]
    col = [-1] * n
    sat = [set() for _ in range(n)]
    for _ in range(n):
        best, bi = None, -1
        for i in range(n):
            if col[i] >= 0:
                continue
            key = (len(sat[i]), len(adj[i]), -i)
            if best is None or key > best:
                best, bi = key, i
        c = 0
        while c in sat[bi]:
            c += 1
        col[bi] = c
        for j in adj[bi]:
            sat[j].add(c)
    return col


def elimination_batches(nbrs, ordering):
    """Clusters grouped into elimination batches: 'natural' = one cluster per
    batch in index order (the left-to-right sweep of Sec. III); 'colored' =
    the colour classes of the near-field graph in increasing colour."""
    n = len(nbrs)
    if ordering == "natural":
        return [[i] for i in range(n)]
    col = greedy_colouring(nbrs)
    return [[i for i in range(n) if col[i] == c] for c in range(max(col) + 1 if n else 0)]


def elimination_order(nbrs, ordering):
    """'natural': left-to-right sweep of Sec. III (i = 1..2^l);
    'colored': colour classes in increasing colour, each in increasing index."""
    n = len(nbrs)
    if ordering == "natural":
        return list(range(n))
    col = greedy_colouring(nbrs)
    return sorted(range(n), key=lambda i: (col[i], i))
