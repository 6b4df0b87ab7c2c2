"""H^2 representation (eq. 2, eq. 3), an exact nested-basis construction, the
H^2 matrix-vector product, and dense assembly of Z_H2 (oracle side).

Representation, in tree order, for levels l0..L:
  * V[c]            leaf cluster basis, #c x k_c, orthonormal columns (eq. 2)
  * T[l][t]         stacked transfer matrix of non-leaf t, (k_t1 + k_t2) x k_t,
                    so that V_t = diag(V_t1, V_t2) T[l][t] (eq. 3)
  * S[l][(t, s)]    coupling of an admissible pair, k_t x k_s:
                    Z_ts ~ V_t S_ts V_s^T (plain transpose, eq. 2)
  * D[(t, s)]       dense inadmissible leaf blocks
The paper builds its H^2 matrices with the method of its refs. [14], [15],
which it does not describe (Sec. VI).  The oracle uses the plain definition of
a nested orthonormal basis at accuracy eps_build:
  leaf t:     V_t = left singular vectors of Z(t, F*(t)) with sigma > eps*sigma_1
  non-leaf t: T_t = left singular vectors of diag(V_t1,V_t2)^H Z(t, F*(t)), same rule
  S_ts = V_t^H Z(t, s) conj(V_s)
where F*(t) holds every column in an admissible block whose row cluster is t
or an ancestor of t.  It costs O(N^2) kernel evaluations: small problems only.
"""
import numpy as np

from . import kernel
from .tree import ClusterTree, Partition


class H2Matrix:
    pass


def _far_columns(tree, part):
    """far[l][t] = list of (level, s) column clusters of F*(t)."""
    L = tree.L
    far = [[[] for _ in range(2 ** l)] for l in range(L + 1)]
    for l in range(L + 1):
        if l > 0:
            for t in range(2 ** l):
                far[l][t] = list(far[l - 1][t // 2])
        for t, s in part.adm[l]:
            far[l][t].append((l, s))
    return far


def eps_rank(sv, eps):
    """Number of singular values kept at relative accuracy eps: sigma > eps * sigma_1
    (sv in descending order; 0 for an empty or zero block)."""
    sv = np.asarray(sv)
    if sv.size == 0 or sv[0] == 0.0:
        return 0
    return int(np.sum(sv > eps * sv[0]))


def build(pts, chi, k, h, leafsize=64, eta=1.0, eps=1e-6, sign=1.0):
    """Exact nested-basis H^2 approximation of Z (see module docstring)."""
    tree = ClusterTree(pts, leafsize)
    part = Partition(tree, eta)
    L, l0 = tree.L, part.l0
    H = H2Matrix()
    H.pts, H.chi, H.k, H.h, H.sign, H.eps = pts, chi, k, h, sign, eps
    H.tree, H.part, H.L, H.l0 = tree, part, L, l0
    far = _far_columns(tree, part)

    def Zb(rows, cols):
        return kernel.entries(pts, chi, rows, cols, k, h, sign)

    def trunc(M):
        if M.shape[1] == 0 or M.shape[0] == 0:
            return np.zeros((M.shape[0], 0), dtype=np.complex128)
        U, sg, _ = np.linalg.svd(M, full_matrices=False)
        return U[:, :eps_rank(sg, eps)].copy()

    full = [dict() for _ in range(L + 1)]  # full basis per level (pins only)
    H.V = {}
    H.T = [dict() for _ in range(L + 1)]
    H.rank = [np.zeros(2 ** l, dtype=np.int64) for l in range(L + 1)]
    for l in range(L, l0 - 1, -1):
        for t in range(2 ** l):
            rows = tree.indices(l, t)
            fc = [tree.indices(lv, s) for lv, s in far[l][t]]
            cols = np.concatenate(fc) if fc else np.zeros(0, dtype=np.int64)
            M = Zb(rows, cols)
            if l == L:
                V = trunc(M)
                H.V[t] = V
                full[l][t] = V
            else:
                V1, V2 = full[l + 1][2 * t], full[l + 1][2 * t + 1]
                W = np.zeros((V1.shape[0] + V2.shape[0], V1.shape[1] + V2.shape[1]), dtype=np.complex128)
                W[:V1.shape[0], :V1.shape[1]] = V1
                W[V1.shape[0]:, V1.shape[1]:] = V2
                Tt = trunc(W.conj().T @ M)
                H.T[l][t] = Tt
                full[l][t] = W @ Tt
            H.rank[l][t] = full[l][t].shape[1]
    H.S = [dict() for _ in range(L + 1)]
    for l in range(l0, L + 1):
        for t, s in part.adm[l]:
            Vt, Vs = full[l][t], full[l][s]
            H.S[l][(t, s)] = Vt.conj().T @ Zb(tree.indices(l, t), tree.indices(l, s)) @ Vs.conj()
    H.D = {}
    for t, s in part.inad[L]:
        H.D[(t, s)] = Zb(tree.indices(L, t), tree.indices(L, s))
    H._full = full
    return H


def full_basis(H, l, t):
    """Explicit nested basis of cluster t at level l, V_t = diag(V_t1,V_t2) T_t."""
    if l == H.L:
        return H.V[t]
    V1, V2 = full_basis(H, l + 1, 2 * t), full_basis(H, l + 1, 2 * t + 1)
    W = np.zeros((V1.shape[0] + V2.shape[0], V1.shape[1] + V2.shape[1]), dtype=np.complex128)
    W[:V1.shape[0], :V1.shape[1]] = V1
    W[V1.shape[0]:, V1.shape[1]:] = V2
    return W @ H.T[l][t]


def dense(H):
    """Z_H2 assembled densely in tree order (for pins at small N)."""
    tree = H.tree
    N = tree.N
    Z = np.zeros((N, N), dtype=np.complex128)
    L = H.L
    for (t, s), Dm in H.D.items():
        a, b = tree.start[L][t], tree.start[L][s]
        Z[a:a + Dm.shape[0], b:b + Dm.shape[1]] = Dm
    for l in range(H.l0, L + 1):
        for (t, s), S in H.S[l].items():
            Vt, Vs = full_basis(H, l, t), full_basis(H, l, s)
            a, b = tree.start[l][t], tree.start[l][s]
            Z[a:a + Vt.shape[0], b:b + Vs.shape[0]] = Vt @ S @ Vs.T
    return Z


def matvec(H, x):
    """y = Z_H2 x for x in tree order (N or N x nrhs): upward pass
    xh_t = V_t^T x_t / T_t^T [xh_t1; xh_t2], coupling yh_t += S_ts xh_s,
    downward pass, and the dense near field (the O(N) H^2 product of Sec. I)."""
    tree, L, l0 = H.tree, H.L, H.l0
    x = np.asarray(x, dtype=np.complex128)
    one = x.ndim == 1
    if one:
        x = x[:, None]
    y = np.zeros_like(x)
    xh = [dict() for _ in range(L + 1)]
    for t in range(2 ** L):
        a = tree.start[L][t]
        xh[L][t] = H.V[t].T @ x[a:a + tree.size[L][t]]
    for l in range(L - 1, l0 - 1, -1):
        for t in range(2 ** l):
            xh[l][t] = H.T[l][t].T @ np.vstack([xh[l + 1][2 * t], xh[l + 1][2 * t + 1]])
    yh = [dict() for _ in range(L + 1)]
    for l in range(l0, L + 1):
        for t in range(2 ** l):
            yh[l][t] = np.zeros((H.rank[l][t], x.shape[1]), dtype=np.complex128)
        for (t, s), S in H.S[l].items():
            yh[l][t] = yh[l][t] + S @ xh[l][s]
    for l in range(l0, L):
        for t in range(2 ** l):
            z = H.T[l][t] @ yh[l][t]
            k1 = H.rank[l + 1][2 * t]
            yh[l + 1][2 * t] = yh[l + 1][2 * t] + z[:k1]
            yh[l + 1][2 * t + 1] = yh[l + 1][2 * t + 1] + z[k1:]
    for t in range(2 ** L):
        a = tree.start[L][t]
        y[a:a + tree.size[L][t]] += H.V[t] @ yh[L][t]
    for (t, s), Dm in H.D.items():
        a, b = tree.start[L][t], tree.start[L][s]
        y[a:a + Dm.shape[0]] += Dm @ x[b:b + Dm.shape[1]]
    return y[:, 0] if one else y
