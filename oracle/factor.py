"""Accuracy-controlled factorization of an H^2 matrix, its explicit inverse,
and forward / backward substitution (oracle side, plain complex128 numpy).

Follows Sec. III (Algorithms 1-4, eqs. 4-35) and Sec. IV (Algorithms 5-6):

  for l = L .. l0:                                   (Algorithm 1)
    for every cluster i at level l, in the elimination order:
      Step 0  basis update from the stored fill-ins, eqs. (16)-(18) / (25)-(27)
      Step 1  complement basis, Q~_i = [V~_i^perp  V~_i], eqs. (4), (19), (28)
      Step 2  Z_cur <- Q_i^H Z_cur conj(Q_i) on row / column i, eq. (5), Alg. 3
      Step 3  partial LU of the first #i - k unknowns, eqs. (9)-(15), Alg. 4
    update couplings (eqs. 20-22, 33), pad transfers (eq. 23), merge (Fig. 2h)
  LU of the final block (Algorithm 1, last line)

Block store.  Every block of the current matrix is kept in the current
coordinates of its row and column clusters: all n_c unknowns before cluster c
is processed at this level, the Q~_c coordinates afterwards, of which only the
trailing k~_c ("kept") stay in Z_cur.  Inadmissible blocks are dense; an
admissible block carries its original coupling S (in the level's incoming
bases) plus one summed fill-in F (eq. 15 and the paragraph after it).

Readings of the paper where it is silent or ambiguous:
  R1 one cluster basis per cluster serves rows and columns (eq. 2); for a
     general, non-symmetric matrix Step 0 adds the column fill-ins
     F_{k,i}^T conj(F_{k,i}) to the row Gram of eq. (16).
  R2 truncation: keep eigenpairs of G_i with lambda > (eps * nu_i)^2, where
     nu_i^2 = sum ||S||_F^2 over the admissible blocks of row and column i at
     this level plus trace(sum F F^H + sum F^T conj(F)).
  R3 a fill-in landing on a pair that the level's partition does not hold
     (it lies inside an ancestor's admissible block) is stored like an
     admissible fill-in ("pushed" block); after the level its kept part is
     carried into the parent pair's fill-in, up to the ancestor level where
     eq. (33) folds it into the coupling.
  R4 Step 1 keeps V~_i verbatim as the last k columns (Householder QR gives
     the complement), so eqs. (7)-(8) hold to round-off.
  R5 partial pivoting inside the m_i x m_i block (largest |z|, lowest row).
  R6 clusters of one colour of the near-field graph are processed as one
     batch (the 'colored' order): Steps 0-1 of every cluster of the batch read
     the state at the start of the batch, Step 2 transforms all block rows of
     the batch and then all block columns, Step 3 forms all partial LUs and
     panels and then all Schur updates.  Clusters of one colour are never near
     neighbours, so this equals a sequential sweep up to the order in which
     fill-ins of non-neighbours are transformed.  'natural' (one cluster per
     batch) is the paper's left-to-right sweep.
  R7 symmetric variant (`symmetric=True`, for a complex-symmetric Z_H2:
     Z^T = Z, S_st = S_ts^T): a block LDL^T elimination.  The Step-2
     transform keeps Z_cur symmetric (Q^H Z conj(Q) with one basis per
     cluster), so only the blocks (a, b) with a <= b are stored and block
     (b, a) is read as the transpose of (a, b).  Eliminating i' with
     F = Z_i'i' (LU with partial pivoting inside F, R5) gives
     Z = [I 0; B F^-1 I] [F 0; 0 S] [I F^-1 B^T; 0 I], S = C - B F^-1 B^T
     with B = Z_(rest) i' = (Z_i' (rest))^T: the factor keeps the raw block
     row Z_i'(rest) once instead of the two panels L^-1 P Z_i'c and
     Z_ci' U^-1, F^-1 is applied through the pivoted LU of F (L^-1 P, then
     U^-1), and S is formed for one triangle of target pairs.  In exact
     arithmetic the Schur complements, hence the rank decisions and the
     solution, equal those of the LU form.
"""
import numpy as np
import scipy.linalg as sla

from . import dense
from .tree import elimination_batches


class ClusterFactor:
    """Factor data of one cluster at one level (the non-identity parts of
    Q_i^l, L_i^l and U_i^l in eq. 34)."""

    __slots__ = ("n", "kt", "m", "Q", "LU", "piv", "Up", "Lp", "Zr")


class LevelFactor:
    __slots__ = ("l", "order", "n", "kt", "cl", "stats")


class Factorization:
    pass


def _linv_p(LU, piv, X):
    """L^{-1} P X with unit lower L from a packed LU."""
    return sla.solve_triangular(LU, X[piv], lower=True, unit_diagonal=True)


def _uinv(LU, X):
    return sla.solve_triangular(LU, X, lower=False)


def _x_uinv(X, LU):
    """X U^{-1} = (U^{-T} X^T)^T."""
    return sla.solve_triangular(LU, X.T, lower=False, trans="T").T


def _transpose(X):
    """Plain transpose: block (b, a) of a complex-symmetric matrix is the
    transpose, not the conjugate transpose, of block (a, b)."""
    return X.T


def _round(X, dtype):
    return X if dtype == np.complex128 else X.astype(dtype).astype(np.complex128)


def ancestor_map(H, l, a, lv):
    """E with V_A(rows of a) = V_a E for the ancestor A of cluster a (level l)
    at level lv < l: the product of the transfer blocks on the path from a up
    to A (eq. 3 applied once per level)."""
    E = np.eye(int(H.rank[l][a]), dtype=np.complex128)
    c = a
    for ll in range(l - 1, lv - 1, -1):
        p = c // 2
        k1 = int(H.rank[ll + 1][2 * p])
        Tp = H.T[ll][p]
        E = E @ (Tp[:k1] if c % 2 == 0 else Tp[k1:])
        c = p
    return E


def _blk(store, a, b, sym):
    """Block (a, b) of a block store; with one-sided storage (`sym`) the
    pairs a > b are the transposed views of the stored (b, a)."""
    return store[(a, b)] if (not sym or a <= b) else store[(b, a)].T


def _has(store, a, b, sym):
    return (a, b) in store if (not sym or a <= b) else (b, a) in store


def factorize(H, eps, ordering="colored", bulk=np.complex128, observe=None, stop_level=None, symmetric=False):
    """Factorize Z_H2 (Algorithm 1).  `bulk`=np.complex64 rounds the Schur /
    LU / transform products to FP32 complex, emulating the mixed-precision
    path; rank decisions (Step 0/1) always run in FP64.  `observe`, if given,
    is called once per Step-0 rank decision with the data it was taken on
    (level, cluster, incoming basis B, the active parts of the row and column
    fill-ins, nu^2, the eigenvalues of G_i in descending order, the threshold
    (eps nu_i)^2, the number r of kept directions and V_add); it only reads
    them.  `stop_level` (Sec. III-C, last paragraph: the factorization may
    stop at a level before l0 is reached): levels L .. stop_level are
    processed, and the remaining matrix of all pairs at stop_level is
    factorized as the final block; a pair that lies inside an ancestor's
    admissible block enters it as pad(E_a S E_b^T) + F, E from
    `ancestor_map` (the coupling in the level's incoming bases, eq. 20).
    `symmetric`: block LDL^T form with one-sided block storage (R7); Z_H2
    must be complex symmetric."""
    tree, part, L, l0 = H.tree, H.part, H.L, H.l0
    sym = bool(symmetric)
    if sym:
        for (t, s_), Dm in H.D.items():
            assert np.allclose(Dm, H.D[(s_, t)].T, rtol=0, atol=1e-12 * (1 + np.abs(Dm).max())), "Z_H2 not symmetric"
    blk = lambda store, a, b: _blk(store, a, b, sym)
    has = lambda store, a, b: _has(store, a, b, sym)
    ls = l0 if stop_level is None else max(l0, min(L, int(stop_level)))
    Fz = Factorization()
    Fz.H, Fz.eps, Fz.ordering, Fz.symmetric = H, eps, ordering, sym
    Fz.levels = []
    # level-L state
    n = np.array(tree.size[L], dtype=np.int64)
    B = {c: H.V[c].copy() for c in range(2 ** L)}
    near = {p: H.D[p].copy() for p in part.inad[L] if not sym or p[0] <= p[1]}
    fill = {}
    for l in range(L, ls - 1, -1):
        near_set = set(part.inad[l])
        adm_set = set(part.adm[l])
        nbrs = part.near_lists(l)
        batches = elimination_batches(nbrs, ordering)
        order = [i for bt in batches for i in bt]
        nc = 2 ** l
        k0 = np.array([B[c].shape[1] for c in range(nc)], dtype=np.int64)
        # sum of ||S||_F^2 over admissible blocks of row and column c (R2)
        snorm2 = np.zeros(nc)
        for (t, s), S in H.S[l].items():
            v = float(np.sum(np.abs(S) ** 2))
            snorm2[t] += v
            snorm2[s] += v
        kt = k0.copy()
        m = np.zeros(nc, dtype=np.int64)
        done = np.zeros(nc, dtype=bool)
        lev = LevelFactor()
        lev.l, lev.order, lev.n = l, order, n.copy()
        lev.cl = {}
        stats = dict(pushed_blocks=0, fill_blocks=0, rank_growth=0)
        fill_rows = {c: [] for c in range(nc)}
        fill_cols = {c: [] for c in range(nc)}
        for (a, b) in fill:
            fill_rows[a].append(b)
            fill_cols[b].append(a)
            if sym:                                             # the (b, a) view
                fill_rows[b].append(a)
                fill_cols[a].append(b)

        def act(c):
            return slice(int(m[c]), int(n[c])) if done[c] else slice(0, int(n[c]))

        for bt in batches:
            # ---- Steps 0 and 1 for every cluster of the batch; they read the
            # state at the start of the batch (R6) ----
            step01 = {}
            for i in bt:
                ni = int(n[i])
                Bi = B[i]
                ki = Bi.shape[1]
                # Step 0: the complement of the incoming basis, from a
                # Householder QR of B_i, gives G_i of eq. (16)/(25) in
                # complement coordinates: G_i = Vp (Vp^H M Vp) Vp^H with
                # M = sum F F^H (+ column side, R1), because I - B B^H = Vp Vp^H.
                # Its eigenvectors Vp U are orthogonal to B_i by construction.
                if ki == 0:
                    Vp = np.eye(ni, dtype=np.complex128)
                else:
                    Qf, _ = np.linalg.qr(Bi, mode="complete")
                    Vp = Qf[:, ki:]
                rows = [(k, blk(fill, i, k)) for k in fill_rows[i]]
                cols = [(k, blk(fill, k, i)) for k in fill_cols[i]]
                Vadd = np.zeros((ni, 0), dtype=np.complex128)
                Vrest = Vp
                if (rows or cols) and ni > ki:
                    M = np.zeros((ni, ni), dtype=np.complex128)
                    for k, Fm in rows:
                        Fa = Fm[:, act(k)]
                        M += Fa @ Fa.conj().T                   # eq. (16) inner sum
                    for k, Fm in cols:
                        Fa = Fm[act(k), :]
                        M += Fa.T @ Fa.conj()                   # column side (R1)
                    Gc = Vp.conj().T @ M @ Vp                   # eq. (16)/(25)
                    Gc = 0.5 * (Gc + Gc.conj().T)
                    w, U = np.linalg.eigh(Gc)                   # eq. (17)/(26)
                    nu2 = snorm2[i] + float(np.real(np.trace(M)))
                    thr = eps * eps * nu2
                    r = int(np.sum(w > thr))
                    if r:
                        Vadd = Vp @ U[:, ::-1][:, :r]           # descending eigenvalues
                        Vrest = Vp @ U[:, ::-1][:, r:]
                        stats["rank_growth"] += r
                    if observe is not None:
                        observe(dict(level=l, cluster=i, B=Bi.copy(), rows=[(k, Fm[:, act(k)].copy()) for k, Fm in rows],
                                     cols=[(k, Fm[act(k), :].copy()) for k, Fm in cols], nu2=nu2, r=r,
                                     Vadd=Vadd.copy(), eig=w[::-1].copy(), thr=thr))
                Bn = np.hstack([Bi, Vadd])                      # eq. (18)/(27)
                # Step 1: complement, Q~_i = [V~^perp, V~] (eq. 19, R4)
                step01[i] = (Bn, np.hstack([Vrest, Bn]))
            for i in bt:
                B[i] = step01[i][0]
                kt[i] = B[i].shape[1]
            # ---- Step 2: Z_cur <- Q_i^H Z_cur conj(Q_i) (eq. 5, Alg. 3):
            # block rows of the batch first, then block columns ----
            # With one-sided storage (R7) the row transform of a view (i, j),
            # j < i, is the column transform of the stored (j, i): every
            # off-diagonal block gets both of its transforms in the row pass,
            # and only the diagonal blocks take the column pass.
            for i in bt:
                Qh = step01[i][1].conj().T
                for j in nbrs[i]:
                    X = blk(near, i, j)
                    cj = slice(0, int(n[i])) if j == i else act(j)
                    X[:, cj] = _round(Qh @ X[:, cj], bulk)
                for kk in fill_rows[i]:
                    X = blk(fill, i, kk)
                    ck = act(kk)
                    X[:, ck] = _round(Qh @ X[:, ck], bulk)
            for i in bt:
                Qb = step01[i][1].conj()
                for j in nbrs[i]:
                    if sym and j != i:
                        continue
                    X = near[(j, i)]
                    cj = slice(0, int(n[i])) if j == i else act(j)
                    X[cj, :] = _round(X[cj, :] @ Qb, bulk)
                for kk in ([] if sym else fill_cols[i]):
                    X = fill[(kk, i)]
                    ck = act(kk)
                    X[ck, :] = _round(X[ck, :] @ Qb, bulk)
            # ---- Step 3: partial LU and panels of the batch, then the Schur
            # updates (Alg. 4) ----
            cfs = {}
            for i in bt:
                ni = int(n[i])
                mi = ni - int(kt[i])
                cf = ClusterFactor()
                cf.n, cf.kt, cf.m, cf.Q = ni, int(kt[i]), mi, step01[i][1]
                cf.Up, cf.Lp, cf.Zr = {}, {}, {}
                cf.LU, cf.piv = None, None
                if mi > 0:
                    LU, piv = dense.lu(near[(i, i)][:mi, :mi])  # eq. (11)
                    LU = _round(LU, bulk)
                    cf.LU, cf.piv = LU, piv
                    if sym:
                        # R7: the raw block row; F^-1 is applied through the
                        # pivoted LU (L^-1 P, then U^-1)
                        for j in nbrs[i]:
                            cs = slice(mi, ni) if j == i else act(j)
                            cf.Zr[j] = (blk(near, i, j)[:mi, cs].copy(), cs)
                        cfs[i] = cf
                        continue
                    for j in nbrs[i]:
                        cs = slice(mi, ni) if j == i else act(j)
                        Uj = _round(_linv_p(LU, piv, near[(i, j)][:mi, cs]), bulk)   # Alg. 4 l.2
                        Lj = _round(_x_uinv(near[(j, i)][cs, :mi], LU), bulk)       # Alg. 4 l.3
                        cf.Up[j] = (Uj, cs)
                        cf.Lp[j] = (Lj, cs)
                cfs[i] = cf
            def target(j, kk, rs, cs, upd):
                if has(near, j, kk):
                    near[(j, kk)][rs, cs] -= upd
                else:                                           # eq. (15): store F_jk
                    if (j, kk) not in fill:
                        fill[(j, kk)] = np.zeros((int(n[j]), int(n[kk])), dtype=np.complex128)
                        fill_rows[j].append(kk)
                        fill_cols[kk].append(j)
                        if sym and j != kk:
                            fill_rows[kk].append(j)
                            fill_cols[j].append(kk)
                        stats["fill_blocks"] += 1
                        if (j, kk) not in adm_set:
                            stats["pushed_blocks"] += 1
                    fill[(j, kk)][rs, cs] -= upd

            for i in bt:
                cf = cfs[i]
                if cf.m == 0 or not sym:
                    continue
                # R7: S_jk -= Z_ji' F^-1 Z_i'k for the stored pairs j <= k
                W = {kk: _round(_uinv(cf.LU, _round(_linv_p(cf.LU, cf.piv, Zk), bulk)), bulk)
                     for kk, (Zk, _) in cf.Zr.items()}
                for j, (Zj, rs) in cf.Zr.items():
                    for kk, (Zk, cs) in cf.Zr.items():
                        if j <= kk:
                            target(j, kk, rs, cs, _round(_transpose(Zj) @ W[kk], bulk))
            for i in bt:
                cf = cfs[i]
                if cf.m == 0 or sym:
                    continue
                for j in nbrs[i]:                               # Alg. 4 l.4, eq. (12)
                    Lj, rs = cf.Lp[j]
                    for kk in nbrs[i]:
                        Uk, cs = cf.Up[kk]
                        target(j, kk, rs, cs, _round(Lj @ Uk, bulk))
            for i in bt:
                m[i] = cfs[i].m
                done[i] = True
                lev.cl[i] = cfs[i]
        lev.kt = kt.copy()
        stats["kt_max"] = int(kt.max()) if nc else 0
        stats["n_max"] = int(n.max()) if nc else 0
        lev.stats = stats
        Fz.levels.append(lev)

        def kept(a, b):
            """Kept (trailing) part of pair (a,b) after the level: the merged
            block of Fig. 2(h); admissible blocks give pad(S) + F (eqs. 20-22)."""
            if (a, b) in near_set:
                return blk(near, a, b)[m[a]:, m[b]:].copy()
            X = np.zeros((int(kt[a]), int(kt[b])), dtype=np.complex128)
            if (a, b) in adm_set:
                S = H.S[l][(a, b)]
                X[:S.shape[0], :S.shape[1]] = S                 # eq. (20)
            elif l > l0:
                # inside the admissible block of an ancestor pair (final block
                # of an early stop): that coupling in the level's bases
                for lv in range(l - 1, l0 - 1, -1):
                    A_, B_ = a >> (l - lv), b >> (l - lv)
                    if (A_, B_) in H.S[lv]:
                        S = ancestor_map(H, l, a, lv) @ H.S[lv][(A_, B_)] @ ancestor_map(H, l, b, lv).T
                        X[:S.shape[0], :S.shape[1]] = S
                        break
            if has(fill, a, b):
                X += blk(fill, a, b)[m[a]:, m[b]:]              # eq. (22)/(33)
            return X

        if l > ls:
            # ---- merge to level l-1 (eq. 23, eq. 24, Fig. 2 g-i) ----
            npar = np.array([kt[2 * p] + kt[2 * p + 1] for p in range(2 ** (l - 1))], dtype=np.int64)
            Bn = {}
            for p in range(2 ** (l - 1)):
                Tp = H.T[l - 1][p]
                c1, c2 = 2 * p, 2 * p + 1
                k1 = int(k0[c1])
                Tn = np.zeros((int(npar[p]), Tp.shape[1]), dtype=np.complex128)
                Tn[:k1] = Tp[:k1]                               # eq. (23) zero padding
                Tn[kt[c1]:kt[c1] + int(k0[c2])] = Tp[k1:]
                Bn[p] = Tn
            near_n = {}
            for p, q in part.inad[l - 1]:
                if sym and p > q:
                    continue
                top = np.hstack([kept(2 * p, 2 * q), kept(2 * p, 2 * q + 1)])
                bot = np.hstack([kept(2 * p + 1, 2 * q), kept(2 * p + 1, 2 * q + 1)])
                near_n[(p, q)] = np.vstack([top, bot])
            near_par = set(part.inad[l - 1])
            fill_n = {}
            for (a, b), Fm in fill.items():
                if (a, b) in adm_set:
                    continue
                pa, pb = a // 2, b // 2
                assert (pa, pb) not in near_par                 # siblings are near: pa != pb
                if (pa, pb) not in fill_n:
                    fill_n[(pa, pb)] = np.zeros((int(npar[pa]), int(npar[pb])), dtype=np.complex128)
                ro = 0 if a % 2 == 0 else int(kt[a - 1])
                co = 0 if b % 2 == 0 else int(kt[b - 1])
                fill_n[(pa, pb)][ro:ro + kt[a], co:co + kt[b]] += Fm[m[a]:, m[b]:]
            n, B, near, fill = npar, Bn, near_n, fill_n
        else:
            # ---- final block: all pairs at level l0, or at the stop level
            # (Alg. 1, last line; Sec. III-C) ----
            off = np.concatenate([[0], np.cumsum(kt)])
            R = np.zeros((off[-1], off[-1]), dtype=np.complex128)
            for a in range(nc):
                for b in range(nc):
                    assert l > l0 or (a, b) in near_set or (a, b) in adm_set
                    R[off[a]:off[a + 1], off[b]:off[b + 1]] = kept(a, b)
            Fz.root_size = int(off[-1])
            Fz.root_off = off
            if off[-1] > 0:
                Fz.root_LU, Fz.root_piv = dense.lu(R)
                Fz.root_LU = _round(Fz.root_LU, bulk)
            else:
                Fz.root_LU, Fz.root_piv = np.zeros((0, 0), dtype=np.complex128), np.zeros(0, dtype=np.int64)
            Fz.root = R
    return Fz


# --------------------------------------------------------------------------
# Solve: Algorithm 5 (forward), root, Algorithm 6 (backward)
# --------------------------------------------------------------------------

def _leaf_split(Fz, v):
    tree, L = Fz.H.tree, Fz.H.L
    return {c: v[tree.start[L][c]:tree.start[L][c] + tree.size[L][c]].copy() for c in range(2 ** L)}


def _merge(lev, vec):
    nc = len(lev.n)
    return {p: np.concatenate([vec[2 * p][lev.n[2 * p] - lev.kt[2 * p]:],
                               vec[2 * p + 1][lev.n[2 * p + 1] - lev.kt[2 * p + 1]:]])
            for p in range(nc // 2)}


def _scatter(lev_child, vec_child, vec_par):
    for p, vp in vec_par.items():
        for c in (2 * p, 2 * p + 1):
            k = int(lev_child.kt[c])
            m = int(lev_child.n[c]) - k
            o = 0 if c % 2 == 0 else int(lev_child.kt[c - 1])
            vec_child[c][m:] = vp[o:o + k]


def _root_split(Fz, lev, y):
    off = Fz.root_off
    out = {}
    for c in range(len(lev.n)):
        out[c] = y[off[c]:off[c + 1]]
    return out


def solve(Fz, b, inverse=None):
    """x = Z^{-1} b via L y = b (Alg. 5, eqs. 36-39) and U x = y (Alg. 6,
    eqs. 40-42); b in tree order (N or N x nrhs).  With `inverse` (from
    `invert`) the same traversal uses the explicit inverse blocks of eq. (35)."""
    b = np.asarray(b, dtype=np.complex128)
    one = b.ndim == 1
    if one:
        b = b[:, None]
    sym = getattr(Fz, "symmetric", False)
    vec = _leaf_split(Fz, b)
    saved = []
    for li, lev in enumerate(Fz.levels):
        for i in lev.order:
            cf = lev.cl[i]
            vec[i] = cf.Q.conj().T @ vec[i]                      # Alg. 5 l.3
            if cf.m > 0 and sym:
                # L of the block LDL^T (R7): y_i' stays, the rest of the
                # vector loses B F^-1 y_i' = Z_i'(rest)^T (F^-1 y_i')
                y = vec[i][:cf.m]
                t = _uinv(cf.LU, _linv_p(cf.LU, cf.piv, y)) if inverse is None else inverse.Finv[li][i] @ y
                for j, (Zj, rs) in cf.Zr.items():
                    vec[j][rs] -= _transpose(Zj) @ t
            elif cf.m > 0:
                if inverse is None:
                    bi = _linv_p(cf.LU, cf.piv, vec[i][:cf.m])   # Alg. 5 l.4, eq. (39)
                else:
                    bi = inverse.Linv[li][i] @ vec[i][:cf.m]
                vec[i][:cf.m] = bi
                for j, (Lj, rs) in cf.Lp.items():
                    vec[j][rs] -= Lj @ bi
        saved.append(vec)
        if li + 1 < len(Fz.levels):
            vec = _merge(lev, vec)                              # P_l
    top = Fz.levels[-1]
    r = np.concatenate([vec[c][top.n[c] - top.kt[c]:] for c in range(len(top.n))]) if Fz.root_size else np.zeros((0, b.shape[1]), dtype=np.complex128)
    if Fz.root_size:
        if inverse is None:
            y = dense.lu_solve(Fz.root_LU, Fz.root_piv, r)
        else:
            y = inverse.Rinv @ r
    else:
        y = r
    par = _root_split(Fz, top, y)
    for li in range(len(Fz.levels) - 1, -1, -1):
        lev = Fz.levels[li]
        vec = saved[li]
        for c, vp in par.items():                               # P_l^T
            k = int(lev.kt[c])
            vec[c][int(lev.n[c]) - k:] = vp
        for i in reversed(lev.order):
            cf = lev.cl[i]
            if cf.m > 0 and sym:
                # D^-1 and L^T (R7): x_i' = F^-1 (y_i' - Z_i'(rest) x_rest)
                t = vec[i][:cf.m].copy()
                if inverse is None:
                    for k_, (Zk, cs) in cf.Zr.items():
                        t -= Zk @ vec[k_][cs]
                    vec[i][:cf.m] = _uinv(cf.LU, _linv_p(cf.LU, cf.piv, t))
                else:
                    t = inverse.Finv[li][i] @ t
                    for k_, (Ub, cs) in inverse.Ub[li][i].items():
                        t += Ub @ vec[k_][cs]
                    vec[i][:cf.m] = t
            elif cf.m > 0:
                if inverse is None:
                    t = vec[i][:cf.m].copy()
                    for k_, (Uk, cs) in cf.Up.items():
                        t -= Uk @ vec[k_][cs]
                    vec[i][:cf.m] = _uinv(cf.LU, t)             # Alg. 6 l.5
                else:
                    t = inverse.Uinv[li][i] @ vec[i][:cf.m]
                    for k_, (Ub, cs) in inverse.Ub[li][i].items():
                        t += Ub @ vec[k_][cs]
                    vec[i][:cf.m] = t
            vec[i] = cf.Q.conj() @ vec[i]                        # Alg. 6 l.6
        if li > 0:
            child = Fz.levels[li - 1]
            par = {}
            for p in range(len(lev.n)):
                v = vec[p]
                k1 = int(child.kt[2 * p])
                par[2 * p] = v[:k1]
                par[2 * p + 1] = v[k1:]
    x = np.concatenate([vec[c] for c in range(len(Fz.levels[0].n))])
    return x[:, 0] if one else x


def solve_adjoint(Fz, r):
    """lambda = Z^{-H} r from the same factors: the adjoints of the solve's
    elementary operations applied in reverse order (U^H then L^H of eq. 34)."""
    r = np.asarray(r, dtype=np.complex128)
    if getattr(Fz, "symmetric", False):
        # Z^T = Z gives Z^-H r = conj(Z^-1 conj(r))
        return np.conj(solve(Fz, np.conj(r)))
    one = r.ndim == 1
    if one:
        r = r[:, None]
    vec = _leaf_split(Fz, r)
    saved = []
    for li, lev in enumerate(Fz.levels):
        for i in lev.order:
            cf = lev.cl[i]
            vec[i] = cf.Q.T @ vec[i]                              # (conj Q)^H
            if cf.m > 0:
                t = sla.solve_triangular(cf.LU, vec[i][:cf.m], lower=False, trans="C")
                vec[i][:cf.m] = t
                for k_, (Uk, cs) in cf.Up.items():
                    vec[k_][cs] -= Uk.conj().T @ t
        saved.append(vec)
        if li + 1 < len(Fz.levels):
            vec = _merge(lev, vec)
    top = Fz.levels[-1]
    if Fz.root_size:
        z = np.concatenate([vec[c][top.n[c] - top.kt[c]:] for c in range(len(top.n))])
        z = sla.solve_triangular(Fz.root_LU, z, lower=False, trans="C")
        z = sla.solve_triangular(Fz.root_LU, z, lower=True, unit_diagonal=True, trans="C")
        y = np.empty_like(z)
        y[Fz.root_piv] = z
    else:
        y = np.zeros((0, r.shape[1]), dtype=np.complex128)
    par = _root_split(Fz, top, y)
    for li in range(len(Fz.levels) - 1, -1, -1):
        lev = Fz.levels[li]
        vec = saved[li]
        for c, vp in par.items():
            k = int(lev.kt[c])
            vec[c][int(lev.n[c]) - k:] = vp
        for i in reversed(lev.order):
            cf = lev.cl[i]
            if cf.m > 0:
                t = vec[i][:cf.m].copy()
                for j, (Lj, rs) in cf.Lp.items():
                    t -= Lj.conj().T @ vec[j][rs]
                t = sla.solve_triangular(cf.LU, t, lower=True, unit_diagonal=True, trans="C")
                u = np.empty_like(t)
                u[cf.piv] = t                                   # P^T
                vec[i][:cf.m] = u
            vec[i] = cf.Q @ vec[i]
        if li > 0:
            child = Fz.levels[li - 1]
            par = {}
            for p in range(len(lev.n)):
                v = vec[p]
                k1 = int(child.kt[2 * p])
                par[2 * p] = v[:k1]
                par[2 * p + 1] = v[k1:]
    x = np.concatenate([vec[c] for c in range(len(Fz.levels[0].n))])
    return x[:, 0] if one else x


class Inverse:
    pass


def invert(Fz):
    """Explicit factor-form inverse of eq. (35): (L_i'i')^{-1} P, (U_i'i')^{-1},
    -(U_i'i')^{-1} U_i'c panels and the inverse of the final block, so that
    applying Z^{-1} needs matrix-vector products only."""
    inv = Inverse()
    inv.Linv, inv.Uinv, inv.Ub, inv.Finv = [], [], [], []
    sym = getattr(Fz, "symmetric", False)
    for lev in Fz.levels:
        Li, Ui, Ubl, Fi = {}, {}, {}, {}
        for i, cf in lev.cl.items():
            if cf.m == 0:
                continue
            if sym:
                # R7: F^-1 and -F^-1 Z_i'c
                Fi[i] = _uinv(cf.LU, _linv_p(cf.LU, cf.piv, np.eye(cf.m, dtype=np.complex128)))
                Ubl[i] = {k: (-Fi[i] @ Zk, cs) for k, (Zk, cs) in cf.Zr.items()}
                continue
            I = np.eye(cf.m, dtype=np.complex128)
            Li[i] = _linv_p(cf.LU, cf.piv, I)
            Ui[i] = _uinv(cf.LU, I)
            Ubl[i] = {k: (-Ui[i] @ Uk, cs) for k, (Uk, cs) in cf.Up.items()}
        inv.Linv.append(Li)
        inv.Uinv.append(Ui)
        inv.Ub.append(Ubl)
        inv.Finv.append(Fi)
    inv.Rinv = dense.lu_solve(Fz.root_LU, Fz.root_piv, np.eye(Fz.root_size, dtype=np.complex128)) if Fz.root_size else None
    return inv


def refine(Fz, b, tol=1e-6, max_iter=20, solve_fn=None):
    """Iterative refinement x += Z^{-1}(b - Z_H2 x) with an FP64 H^2 matvec."""
    from .h2 import matvec
    solve_fn = solve_fn or (lambda v: solve(Fz, v))
    x = solve_fn(b)
    nb = np.linalg.norm(b)
    hist = []
    for _ in range(max_iter + 1):
        r = b - matvec(Fz.H, x)
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if rel <= tol or len(hist) > max_iter:
            break
        x = x + solve_fn(r)
    return x, hist
