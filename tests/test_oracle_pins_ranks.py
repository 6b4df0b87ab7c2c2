"""Pins of the oracle's rank decisions and of its mixed-precision emulation
against things other than the oracle's own code path:

  * the growth of the eps-rank of an admissible interaction with electric
    size that the paper states (Sec. I; Sec. V, eqs. 43-44), on blocks of the
    oracle's kernel with the oracle's construction rule;
  * Step 0's truncation (eqs. 16-17, reading R2) against an explicit SVD of
    the projected fill-in blocks (a different route to the same numbers);
  * the complex64-bulk emulation (the mixed path's oracle) against LAPACK's
    complex64 LU of the same matrix and against refinement to the FP64
    solution.
"""
import math

import numpy as np

from oracle import factor, h2, kernel, tree
from paper_1703_06155_gb300 import inputs

from _problems import factorization, h2_dense, h2_problem

K = 2.0 * math.pi


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cube(m, h, x0):
    c = (np.arange(m) + 0.5) * h
    g = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    return g + np.array([x0, 0.0, 0.0])


def test_rank_grows_linearly_with_electric_size():
    # Two cubes of side a (points at h = lambda / 8) whose bounding spheres
    # touch: the pair is admissible by eq. (1) with eta = 1 (the oracle's own
    # tree and partition decide it).  The eps-rank of their interaction,
    # counted by the construction's rule (sigma > eps sigma_1), must grow
    # with a, affinely ("linearly with the electric size", Sec. I), and
    # slower than the area (a^2) or volume (a^3) of the cluster.
    h, eps = 1.0 / 8.0, 1e-4
    sides, ranks = [], []
    for m in (4, 6, 8, 10, 12, 16):
        p1 = _cube(m, h, 0.0)
        r = np.max(np.linalg.norm(p1 - p1.mean(axis=0), axis=1))
        pts = np.vstack([p1, _cube(m, h, 2.0 * r * (1.0 + 1e-12))])
        T = tree.ClusterTree(pts, len(p1))
        P = tree.Partition(T, 1.0)
        assert T.L == 1 and (0, 1) in P.adm[1], "the two cubes must form one admissible pair"
        Z = kernel.entries(pts, np.ones(len(pts)), T.indices(1, 0), T.indices(1, 1), K, h)
        sides.append(m * h)
        ranks.append(h2.eps_rank(np.linalg.svd(Z, compute_uv=False), eps))
    a, k = np.array(sides), np.array(ranks, dtype=float)
    assert np.all(np.diff(k) >= 0), ranks
    big = a >= 1.0
    slope, icpt = np.polyfit(a[big], k[big], 1)
    fit = slope * a[big] + icpt
    r2 = 1.0 - np.sum((k[big] - fit) ** 2) / np.sum((k[big] - k[big].mean()) ** 2)
    expo = np.polyfit(np.log(a[big]), np.log(k[big]), 1)[0]
    print("ranks", dict(zip(sides, ranks)), "affine slope %.2f / lambda, R^2 %.4f, log-log exponent %.3f"
          % (slope, r2, expo))
    assert slope > 0 and r2 >= 0.97, (slope, r2)
    grow = k[a == 2.0][0] / k[a == 1.0][0]
    assert 1.2 <= grow <= 2.0, grow  # doubling a: rank grows, at most doubles (area law: x4)


def test_step0_truncation_matches_svd_of_projected_fill_ins():
    # Reading R2 of eq. (17): keep the directions of G_i = Pi (sum F F^H +
    # sum F^T conj F) Pi with lambda > (eps nu_i)^2, Pi the projector onto the
    # complement of the incoming basis, nu_i^2 = sum ||S||_F^2 over the
    # admissible blocks of row and column i + ||F||_F^2.  The eigenvalues of
    # G_i are the squared singular values of Pi W, W = [F_row ..., F_col^T ...],
    # so an SVD of Pi W (with Pi applied as I - B B^H) must give the same count
    # and span the same directions.
    eps = 1e-4
    H = h2_problem(12, 64, eps)
    recs = []
    factor.factorize(H, eps, "colored", observe=recs.append)
    assert len(recs) > 20
    checked = grown = 0
    for rec in recs:
        l, i, B = rec["level"], rec["cluster"], rec["B"]
        blocks = [F for _, F in rec["rows"]] + [F.T for _, F in rec["cols"]]
        W = np.hstack(blocks)
        PW = W - B @ (B.conj().T @ W)
        sv = np.linalg.svd(PW, compute_uv=True)
        U, s = sv[0], sv[1]
        snorm2 = sum(float(np.sum(np.abs(S) ** 2)) for (t, u), S in H.S[l].items() if t == i or u == i)
        nu2 = snorm2 + float(np.sum(np.abs(W) ** 2))
        assert abs(rec["nu2"] - nu2) <= 1e-10 * nu2
        thr = eps * math.sqrt(nu2)
        if np.any(np.abs(s - thr) <= 1e-6 * thr):
            continue  # a singular value at the threshold: either decision is right
        r = int(np.sum(s > thr))
        assert rec["r"] == r, (l, i, rec["r"], r)
        if r:
            Va = rec["Vadd"]
            # same span: the kept directions lie in the top-r left singular space
            assert np.linalg.norm(Va - U[:, :r] @ (U[:, :r].conj().T @ Va)) < 1e-6
            assert np.linalg.norm(B.conj().T @ Va) < 1e-12  # orthogonal to the incoming basis
            grown += 1
        checked += 1
    assert checked >= 0.9 * len(recs) and grown > 5, (checked, grown, len(recs))


def test_complex64_bulk_emulation():
    # eps_fill = 0 makes the factorization an exact block LU of Z_H2; with the
    # bulk rounded to complex64 its solution error must be that of a complex64
    # LU of the same matrix (LAPACK's cgesv through numpy), and FP64
    # refinement must recover the complex128 solution.
    H = h2_problem(12, 64, 1e-6)
    Zd = h2_dense(12, 64, 1e-6)
    b = inputs.rhs_gaussian(H.tree.N, 2, 13)
    bt = b[H.tree.perm]
    xe = np.linalg.solve(Zd, bt)
    Fz = factor.factorize(H, 0.0, "colored", bulk=np.complex64)
    e32 = rel(factor.solve(Fz, bt), xe)
    el = rel(np.linalg.solve(Zd.astype(np.complex64), bt.astype(np.complex64)).astype(np.complex128), xe)
    e64 = rel(factor.solve(factorization(12, 64, 1e-6, 0.0, "colored"), bt), xe)
    print("complex64 bulk %.2e, LAPACK complex64 LU %.2e, complex128 bulk %.2e" % (e32, el, e64))
    assert e64 < 1e-11
    assert el > 1e3 * e64  # a complex64 LU is far from complex128 accuracy here
    assert el / 30 <= e32 <= 30 * el, (e32, el)
    x, hist = factor.refine(Fz, bt, tol=1e-13, max_iter=30)
    assert hist[-1] <= 1e-13 and rel(x, xe) < 1e-10, (hist, rel(x, xe))
    # with eps_fill = eps as well: the emulated mixed path refines to the same solution
    Fm = factor.factorize(H, 1e-6, "colored", bulk=np.complex64)
    x, hist = factor.refine(Fm, bt, tol=1e-13, max_iter=30)
    assert hist[-1] <= 1e-13 and rel(x, xe) < 1e-10, (hist, rel(x, xe))


def test_early_stop_levels():
    # Sec. III-C, last paragraph: the factorization may stop at any level
    # above l0, the rest being factorized as one dense block.  With
    # eps_fill = 0 every stop level gives an exact block LU of Z_H2; with
    # eps_fill > 0 the residual stays at the eps level and decreases as the
    # stop level moves towards the leaves (fewer truncations), and the final
    # block grows.
    eps = 1e-6
    H = h2_problem(8, 16, eps)  # 512 points, leaf 16: five levels below l0 = 3
    Zd = h2_dense(8, 16, eps)
    b = inputs.rhs_gaussian(H.tree.N, 2, 17)[H.tree.perm]
    xe = np.linalg.solve(Zd, b)
    sizes, res = [], []
    for ls in range(H.l0, H.L + 1):
        F0 = factor.factorize(H, 0.0, "colored", stop_level=ls)
        assert len(F0.levels) == H.L - ls + 1
        assert rel(factor.solve(F0, b), xe) < 1e-11, ls
        Fe = factor.factorize(H, eps, "colored", stop_level=ls)
        x = factor.solve(Fe, b)
        res.append(np.linalg.norm(Zd @ x - b) / np.linalg.norm(b))
        sizes.append(Fe.root_size)
        # the explicit inverse (eq. 35) and the adjoint traversal work on the same factors
        xi = factor.solve(Fe, b, inverse=factor.invert(Fe))
        assert rel(xi, x) < 1e-12
        xa = factor.solve_adjoint(Fe, b)
        assert rel(xa, np.linalg.solve(Zd.conj().T, b)) < 10 * eps
    assert max(res) <= 10 * eps and res[-1] <= res[0], res
    assert all(s1 >= s0 for s0, s1 in zip(sizes, sizes[1:])) and sizes[-1] > sizes[0], sizes


def test_rod_ranks_stay_bounded():
    # Sec. VI-B: a rod (fixed 0.4 x 0.4 wavelength cross-section, growing
    # length) has 1-D rank characteristics: the rank does not grow with the
    # electric length, which is what makes the solver strictly O(N) there.
    # The oracle's construction on rods of 6, 12 and 24 wavelengths (h = 0.1):
    # the largest rank at each distance from the leaves is the same to within
    # a few directions, whatever the length.
    eps = 1e-4
    tops = []
    for length in (6.0, 12.0, 24.0):
        pts = inputs.rod_points(length, 0.1)
        Hm = h2.build(pts, inputs.chi_uniform(len(pts), 1.54), K, 0.1, leafsize=64, eps=eps)
        per = [int(Hm.rank[l].max()) for l in range(Hm.L, Hm.l0 - 1, -1)]  # leaf level first
        tops.append(per)
    print("rod ranks by level from the leaves:", tops)
    depth = min(len(t) for t in tops)
    for d in range(depth - 1):  # the top level of the shortest rod has the smallest far field
        vals = [t[d] for t in tops]
        assert max(vals) - min(vals) <= max(3, 0.1 * max(vals)), (d, vals)
    assert max(max(t) for t in tops) <= 1.15 * max(tops[0])
