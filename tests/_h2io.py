"""Conversion of the oracle's H^2 matrix into the host-array layout that the
C ABI's h2_load takes (test infrastructure)."""
import numpy as np


def _cm(a):
    return np.asarray(a, dtype=np.complex128).ravel(order="F")


def oracle_to_rep(H, dscale=None):
    L, l0, tree, part = H.L, H.l0, H.tree, H.part
    rank = np.concatenate([H.rank[l] for l in range(l0, L + 1)]).astype(np.int64)
    V = np.concatenate([_cm(H.V[c]) for c in range(2 ** L)] + [np.zeros(0, np.complex128)])
    T = np.concatenate([_cm(H.T[l][c]) for l in range(l0, L) for c in range(2 ** l)] + [np.zeros(0, np.complex128)])
    n_adm = np.array([len(part.adm[l]) for l in range(l0, L + 1)], dtype=np.int64)
    adm = np.array([x for l in range(l0, L + 1) for p in part.adm[l] for x in p], dtype=np.int64)
    S = np.concatenate([_cm(H.S[l][p]) for l in range(l0, L + 1) for p in part.adm[l]] + [np.zeros(0, np.complex128)])
    near = np.array([x for p in part.inad[L] for x in p], dtype=np.int64)
    D = np.concatenate([_cm(H.D[p]) for p in part.inad[L]])
    return dict(N=tree.N, L=L, l0=l0, perm=tree.perm.astype(np.int64), leaf_size=np.asarray(tree.size[L], np.int64),
                rank=rank, V=V, T=T, n_adm=n_adm, adm=adm, S=S, near=near, D=D, dscale=dscale)


def to_tree(H, x):
    return np.asarray(x)[H.tree.perm]


def from_tree(H, y):
    out = np.empty_like(y)
    out[H.tree.perm] = y
    return out


def dense_from_rep(r):
    """Assemble Z_H2 (tree order) from the h2_load layout, independently of
    both the oracle and the library."""
    L, l0 = r["L"], r["l0"]
    ranks, o = {}, 0
    for l in range(l0, L + 1):
        ranks[l] = r["rank"][o:o + 2 ** l]
        o += 2 ** l
    sizes = {L: r["leaf_size"]}
    for l in range(L - 1, -1, -1):
        sizes[l] = sizes[l + 1][0::2] + sizes[l + 1][1::2]
    starts = {l: np.concatenate([[0], np.cumsum(sizes[l])[:-1]]) for l in sizes}
    full, o = {}, 0
    for c in range(2 ** L):
        cnt = sizes[L][c] * ranks[L][c]
        full[(L, c)] = r["V"][o:o + cnt].reshape(ranks[L][c], sizes[L][c]).T
        o += cnt
    Tm, o = {}, 0
    for l in range(l0, L):
        for c in range(2 ** l):
            k1, k2 = ranks[l + 1][2 * c], ranks[l + 1][2 * c + 1]
            cnt = (k1 + k2) * ranks[l][c]
            Tm[(l, c)] = r["T"][o:o + cnt].reshape(ranks[l][c], k1 + k2).T
            o += cnt
    for l in range(L - 1, l0 - 1, -1):
        for c in range(2 ** l):
            A1, A2 = full[(l + 1, 2 * c)], full[(l + 1, 2 * c + 1)]
            W = np.zeros((A1.shape[0] + A2.shape[0], A1.shape[1] + A2.shape[1]), complex)
            W[:A1.shape[0], :A1.shape[1]] = A1
            W[A1.shape[0]:, A1.shape[1]:] = A2
            full[(l, c)] = W @ Tm[(l, c)]
    N = r["N"]
    Z = np.zeros((N, N), complex)
    adm = r["adm"].reshape(-1, 2)
    o = so = 0
    for i, l in enumerate(range(l0, L + 1)):
        for q in range(r["n_adm"][i]):
            t, s = adm[o]
            o += 1
            cnt = ranks[l][t] * ranks[l][s]
            S = r["S"][so:so + cnt].reshape(ranks[l][s], ranks[l][t]).T
            so += cnt
            Z[starts[l][t]:starts[l][t] + sizes[l][t], starts[l][s]:starts[l][s] + sizes[l][s]] = \
                full[(l, t)] @ S @ full[(l, s)].T
    do = 0
    for t, s in r["near"].reshape(-1, 2):
        cnt = sizes[L][t] * sizes[L][s]
        Z[starts[L][t]:starts[L][t] + sizes[L][t], starts[L][s]:starts[L][s] + sizes[L][s]] = \
            r["D"][do:do + cnt].reshape(sizes[L][s], sizes[L][t]).T
        do += cnt
    return Z, full
