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
