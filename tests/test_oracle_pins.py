"""Pins of the CPU oracle against things other than itself: closed forms,
numerical quadrature, LAPACK, brute-force dense algebra, exact identities of
the paper (eqs. 7-8, 34-35), the eps_fill -> 0 limit and the eps sweep."""
import math

import numpy as np
import pytest
import scipy.integrate as si

from oracle import dense, factor, h2, kernel, tree
from paper_1703_06155_gb300 import inputs

from _problems import H, K, factorization, h2_dense, h2_problem
from _h2io import from_tree, to_tree

# --------------------------------------------------------------- kernel ----


def test_self_term_series():
    # (1 + jx) e^{-jx} - 1 = x^2/2 - j x^3/3 - x^4/8 + j x^5/30 + O(x^6)
    for h in (1 / 16, 1 / 64, 1 / 256):
        x = K * kernel.ball_radius(h)
        ser = x ** 2 / 2 - 1j * x ** 3 / 3 - x ** 4 / 8 + 1j * x ** 5 / 30
        assert abs(kernel.self_term(K, h) - ser) <= 2 * x ** 6


def test_self_term_quadrature():
    # k^2 int_0^a (e^{-jkr} / (4 pi r)) 4 pi r^2 dr, integrated numerically
    a = kernel.ball_radius(H)
    re = si.quad(lambda r: K * K * r * math.cos(K * r), 0, a, epsabs=1e-15)[0]
    im = si.quad(lambda r: -K * K * r * math.sin(K * r), 0, a, epsabs=1e-15)[0]
    ref = 0.029234 - 0.004791j  # value at h = 1/16, k = 2 pi
    assert abs(kernel.self_term(K, H) - (re + 1j * im)) < 1e-13
    assert abs(kernel.self_term(K, H) - ref) < 1e-6


def test_offdiagonal_kernel_integrates_to_self_term():
    # Summing the off-diagonal entries over a fine grid filling the
    # equal-volume ball approximates k^2 int G dV, i.e. the closed form.
    a = kernel.ball_radius(H)
    m = 41
    d = 2 * a / m
    c = (np.arange(m) - (m - 1) / 2) * d
    g = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    inside = np.linalg.norm(g, axis=1) <= a
    pts = np.vstack([[0.0, 0.0, 0.0], g[inside & (np.linalg.norm(g, axis=1) > 0)]])
    chi = np.ones(len(pts))
    row = kernel.entries(pts, chi, np.array([0]), np.arange(1, len(pts)), K, d)
    approx = row.sum()
    exact = kernel.self_term(K, H)
    # missing central cell contributes about k^2 * (3/(4pi))^(2/3) d^2 / 2
    assert abs(approx - exact) / abs(exact) < 0.05
    assert np.sign(approx.imag) == np.sign(exact.imag)


def test_green_function_solves_helmholtz():
    # (nabla^2 + k^2) G = 0 away from the source, by central differences
    p0 = np.array([[0.0, 0.0, 0.0]])
    x = np.array([0.37, -0.21, 0.52])
    dl = 1e-3
    offs = [np.zeros(3)] + [s * dl * e for e in np.eye(3) for s in (1, -1)]
    pts = np.vstack([p0] + [x + o for o in offs])
    g = kernel.entries(pts, np.ones(len(pts)), np.array([0]), np.arange(1, len(pts)), K, 1.0)[0]
    lap = (g[1:].sum() - 6 * g[0]) / dl ** 2
    assert abs(lap + K * K * g[0]) / abs(K * K * g[0]) < 1e-4


def test_matrix_is_symmetric_and_similar_to_A():
    pts = inputs.grid_points(6, H)
    N = len(pts)
    chi = inputs.chi_random_cells(N, 5)
    idx = np.arange(N)
    Z = kernel.entries(pts, chi, idx, idx, K, H)
    A = kernel.dense_A(pts, chi, K, H)
    D = np.sqrt(chi)
    assert np.allclose(Z, Z.T, atol=1e-15)
    assert np.allclose(Z, D[:, None] * A / D[None, :], atol=1e-14)


# ------------------------------------------------------- tree/partition ----


@pytest.mark.parametrize("n,leaf", [(8, 16), (12, 64), (16, 64)])
def test_partition_covers_each_entry_once(n, leaf):
    pts = inputs.grid_points(n, H)
    T = tree.ClusterTree(pts, leaf)
    P = tree.Partition(T, 1.0)
    N = T.N
    assert max(T.size[T.L]) <= leaf and min(T.size[T.L]) >= leaf // 2
    for l in range(T.L + 1):
        assert len(T.size[l]) == 2 ** l and T.size[l].max() - T.size[l].min() <= 1
    mark = np.zeros((N, N), dtype=np.int32)
    for l in range(T.L + 1):
        for t, s in P.adm[l]:
            a, b = T.start[l][t], T.start[l][s]
            mark[a:a + T.size[l][t], b:b + T.size[l][s]] += 1
            d = np.linalg.norm(T.centre[l][t] - T.centre[l][s])
            assert d >= T.radius[l][t] + T.radius[l][s]
    for t, s in P.inad[T.L]:
        a, b = T.start[T.L][t], T.start[T.L][s]
        mark[a:a + T.size[T.L][t], b:b + T.size[T.L][s]] += 1
    assert (mark == 1).all()
    assert sorted(T.perm.tolist()) == list(range(N))


def test_colouring_is_proper():
    pts = inputs.grid_points(16, H)
    T = tree.ClusterTree(pts, 64)
    P = tree.Partition(T, 1.0)
    for l in range(P.l0, T.L + 1):
        nb = P.near_lists(l)
        col = tree.greedy_colouring(nb)
        for i in range(len(nb)):
            for j in nb[i]:
                assert j == i or col[i] != col[j]


# --------------------------------------------------------- construction ----


@pytest.mark.parametrize("n,leaf,eps", [(8, 16, 1e-6), (12, 64, 1e-6), (12, 64, 1e-3)])
def test_h2_approximates_dense_matrix(n, leaf, eps):
    Hm = h2_problem(n, leaf, eps)
    Zh = h2_dense(n, leaf, eps)
    idx = Hm.tree.perm
    Z = kernel.entries(Hm.pts, Hm.chi, idx, idx, K, H)
    assert np.linalg.norm(Zh - Z) / np.linalg.norm(Z) < 10 * eps
    for l in range(Hm.l0, Hm.L + 1):
        for (t, s), S in Hm.S[l].items():
            # symmetric matrix -> S_st = S_ts^T
            assert np.allclose(Hm.S[l][(s, t)], S.T, atol=1e-12 * np.abs(S).max())
    for c, V in Hm.V.items():
        assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-13
    for l in range(Hm.l0, Hm.L):
        for t, T in Hm.T[l].items():
            assert np.abs(T.conj().T @ T - np.eye(T.shape[1])).max() < 1e-13


def test_matvec_matches_dense_assembly():
    Hm = h2_problem(12, 64, 1e-6)
    Zh = h2_dense(12, 64, 1e-6)
    x = inputs.rhs_gaussian(Hm.tree.N, 3, 7)
    y = h2.matvec(Hm, x)
    assert np.linalg.norm(y - Zh @ x) / np.linalg.norm(Zh @ x) < 1e-14


# ------------------------------------------------------------ dense LU ----


def test_dense_lu_against_lapack():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((60, 60)) + 1j * rng.standard_normal((60, 60))
    b = rng.standard_normal(60) + 1j * rng.standard_normal(60)
    assert np.allclose(dense.solve(A, b), np.linalg.solve(A, b), atol=1e-12)
    assert np.allclose(dense.inverse(A), np.linalg.inv(A), atol=1e-12)
    LU, piv = dense.lu(A)
    L = np.tril(LU, -1) + np.eye(60)
    U = np.triu(LU)
    assert np.allclose(A[piv], L @ U, atol=1e-12)
    assert (np.abs(np.tril(LU, -1)) <= 1 + 1e-12).all()  # partial pivoting bound


# ------------------------------------------------------- factorization ----


@pytest.mark.parametrize("ordering", ["colored", "natural"])
def test_eps_zero_is_exact_block_lu(ordering):
    # eps_fill -> 0 keeps every fill-in direction: the only approximation of
    # the method vanishes (Sec. V-A) and Z_H2 = LU exactly (eq. 34).
    Fz = factorization(12, 64, 1e-6, 0.0, ordering)
    Zh = h2_dense(12, 64, 1e-6)
    b = inputs.rhs_gaussian(Fz.H.tree.N, 2, 11)
    x = factor.solve(Fz, b)
    xe = np.linalg.solve(Zh, b)
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) < 1e-11
    lam = factor.solve_adjoint(Fz, b)
    le = np.linalg.solve(Zh.conj().T, b)
    assert np.linalg.norm(lam - le) / np.linalg.norm(le) < 1e-11


def test_complement_identities_eq7_eq8():
    Fz = factorization(12, 64, 1e-6, 1e-6, "colored")
    Hm = Fz.H
    leaf = Fz.levels[0]
    for i, cf in leaf.cl.items():
        Q = cf.Q
        assert np.abs(Q.conj().T @ Q - np.eye(cf.n)).max() < 1e-13
        V = Hm.V[i]
        k0 = V.shape[1]
        # V~ = [V, V_add] sits verbatim in the last k~ columns (eq. 18, 19)
        assert np.abs(Q[:, cf.m:cf.m + k0] - V).max() < 1e-14
        # eq. (7): Q~^H V = [0; I]; eq. (8): V^T conj(Q~) = [0 I]
        QV = Q.conj().T @ V
        assert np.abs(QV[:cf.m]).max() < 1e-13
        assert np.abs(QV[cf.m:cf.m + k0] - np.eye(k0)).max() < 1e-13
        VQ = V.T @ Q.conj()
        assert np.abs(VQ[:, :cf.m]).max() < 1e-13


def test_residual_tracks_eps():
    # eps_build = eps_fill = eps, as in the configured workloads; the residual
    # is measured against the input H^2 matrix (Sec. VI), so only the
    # factorization's truncation (eqs. 17, 26) contributes.
    b = inputs.rhs_gaussian(12 ** 3, 1, 0)[:, 0]
    eps_list = [1e-3, 1e-5, 1e-7]
    res = []
    for e in eps_list:
        Zh = h2_dense(12, 64, e)
        Fz = factorization(12, 64, e, e, "colored")
        x = factor.solve(Fz, b)
        res.append(np.linalg.norm(Zh @ x - b) / np.linalg.norm(b))
    assert res[0] > res[1] > res[2]
    slope = np.polyfit(np.log10(eps_list), np.log10(res), 1)[0]
    assert 0.7 <= slope <= 1.3, (res, slope)
    assert all(r < 10 * e for r, e in zip(res, eps_list))


def test_colored_and_natural_agree_to_eps():
    Zh = h2_dense(12, 64, 1e-6)
    b = inputs.rhs_gaussian(Zh.shape[0], 1, 0)[:, 0]
    xc = factor.solve(factorization(12, 64, 1e-6, 1e-6, "colored"), b)
    xn = factor.solve(factorization(12, 64, 1e-6, 1e-6, "natural"), b)
    xe = np.linalg.solve(Zh, b)
    assert np.linalg.norm(xc - xn) / np.linalg.norm(xe) < 1e-5


def test_inverse_apply_matches_solve_and_dense_inverse():
    Fz = factorization(12, 64, 1e-6, 0.0, "colored")
    inv = factor.invert(Fz)
    b = inputs.rhs_gaussian(Fz.H.tree.N, 2, 5)
    x = factor.solve(Fz, b)
    xi = factor.solve(Fz, b, inverse=inv)
    assert np.linalg.norm(xi - x) / np.linalg.norm(x) < 1e-12
    Zi = dense.inverse(h2_dense(12, 64, 1e-6))
    assert np.linalg.norm(xi - Zi @ b) / np.linalg.norm(x) < 1e-11


def test_refinement_converges():
    Fz = factorization(12, 64, 1e-6, 1e-4, "colored")
    b = inputs.rhs_gaussian(Fz.H.tree.N, 1, 0)[:, 0]
    x, hist = factor.refine(Fz, b, tol=1e-12, max_iter=10)
    assert hist[-1] <= 1e-12 and len(hist) <= 6
    Zh = h2_dense(12, 64, 1e-6)
    assert np.linalg.norm(Zh @ x - b) / np.linalg.norm(b) < 1e-11


def test_trivial_cases():
    # zero contrast: Z = I, so x = b exactly
    pts = inputs.grid_points(8, H)
    N = len(pts)
    Hm = h2.build(pts, np.zeros(N), K, H, leafsize=16, eps=1e-6)
    Fz = factor.factorize(Hm, 1e-6)
    b = inputs.rhs_gaussian(N, 1, 1)[:, 0]
    assert np.allclose(factor.solve(Fz, b), b, atol=1e-14)
    # huge eta: no admissible block, plain block LU of the dense matrix
    from oracle.tree import ClusterTree, Partition
    T = ClusterTree(pts, 16)
    P = Partition(T, 1e9)
    assert sum(len(a) for a in P.adm) == 0


@pytest.mark.parametrize("N", [1, 2, 7, 65, 129])
def test_degenerate_sizes(N):
    # one point (never admissible with itself), fewer points than a leaf (the
    # whole matrix is one near-field block), one point past a leaf and a
    # ragged two-level tree: exact at eps = 0, within eps of the dense solve
    from oracle import kernel
    from oracle.tree import ClusterTree, Partition
    pts = np.ascontiguousarray(inputs.grid_points(6, H)[:N])
    chi = inputs.chi_uniform(N, 3.0)
    T = ClusterTree(pts, 64)
    P = Partition(T, 1.0)
    assert all((t, t) not in P.adm[l] for l in range(T.L + 1) for t in range(2 ** l))
    idx = np.arange(N)
    Z = kernel.entries(pts, chi, idx, idx, K, H)
    b = inputs.rhs_gaussian(N, 1, 3)[:, 0]
    xe = np.linalg.solve(Z, b)
    for eps, tol in ((0.0, 1e-12), (1e-6, 1e-5)):
        Hm = h2.build(pts, chi, K, H, leafsize=64, eps=max(eps, 1e-12))
        Fz = factor.factorize(Hm, eps)
        x = from_tree(Hm, factor.solve(Fz, to_tree(Hm, b)))
        assert np.linalg.norm(x - xe) <= tol * np.linalg.norm(xe), (eps, np.linalg.norm(x - xe))


# ------------------------------------- block LDL^T (symmetric) variant ----


@pytest.mark.parametrize("ordering", ["colored", "natural"])
def test_ldlt_eps_zero_is_exact(ordering):
    # eps_fill = 0: the block LDL^T of the symmetric Z_H2 with one-sided block
    # storage is exact (Z = L D L^T), like the LU form (eq. 34); the adjoint
    # (Z^-H = conj Z^-1 conj) and the factor-form inverse follow it
    Hm = h2_problem(12, 64, 1e-6)
    Zh = h2_dense(12, 64, 1e-6)
    Fz = factor.factorize(Hm, 0.0, ordering, symmetric=True)
    b = inputs.rhs_gaussian(Hm.tree.N, 2, 11)
    xe = np.linalg.solve(Zh, b)
    assert np.linalg.norm(factor.solve(Fz, b) - xe) / np.linalg.norm(xe) < 1e-11
    le = np.linalg.solve(Zh.conj().T, b)
    assert np.linalg.norm(factor.solve_adjoint(Fz, b) - le) / np.linalg.norm(le) < 1e-11
    xi = factor.solve(Fz, b, inverse=factor.invert(Fz))
    assert np.linalg.norm(xi - xe) / np.linalg.norm(xe) < 1e-11


def test_ldlt_matches_lu_form_and_halves_the_blocks():
    # eps_fill > 0: the two forms compute the same Schur complements in exact
    # arithmetic, so every Step-0 decision (per-cluster kept ranks) and the
    # solution agree to rounding; the symmetric form stores one block of each
    # off-diagonal pair, half the fill-in blocks of the LU form
    Hm = h2_problem(12, 64, 1e-6)
    b = inputs.rhs_gaussian(Hm.tree.N, 1, 4)[:, 0]
    for eps in (1e-6, 1e-4):
        Flu = factorization(12, 64, 1e-6, eps, "colored")
        Fs = factor.factorize(Hm, eps, "colored", symmetric=True)
        for a, c in zip(Flu.levels, Fs.levels):
            assert np.array_equal(a.kt, c.kt), (a.l, a.kt, c.kt)
            assert 2 * c.stats["fill_blocks"] == a.stats["fill_blocks"]
        x1, x2 = factor.solve(Flu, b), factor.solve(Fs, b)
        assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-12


def test_ldlt_early_stop_and_percell_contrast_exact():
    # per-cell contrast keeps Z = D^1/2 A D^-1/2 symmetric (R12), and an early
    # stop (Sec. III-C) assembles its final block from the one-sided store:
    # both stay exact at eps_fill = 0
    for Hm, Zh, stop in ((h2_problem(12, 64, 1e-6, percell_seed=3), h2_dense(12, 64, 1e-6, percell_seed=3), None),
                         (h2_problem(12, 64, 1e-6), h2_dense(12, 64, 1e-6), 4)):
        Fz = factor.factorize(Hm, 0.0, "colored", stop_level=stop, symmetric=True)
        b = inputs.rhs_gaussian(Hm.tree.N, 1, 7)[:, 0]
        xe = np.linalg.solve(Zh, b)
        assert np.linalg.norm(factor.solve(Fz, b) - xe) / np.linalg.norm(xe) < 1e-11


def test_ldlt_refinement_from_complex64_bulk():
    # the mixed-precision emulation (complex64 bulk) of the symmetric form,
    # refined with the FP64 H^2 matvec, reaches the dense solution
    Hm = h2_problem(12, 64, 1e-6)
    Zh = h2_dense(12, 64, 1e-6)
    Fz = factor.factorize(Hm, 1e-6, "colored", bulk=np.complex64, symmetric=True)
    b = inputs.rhs_gaussian(Hm.tree.N, 1, 6)[:, 0]
    x, hist = factor.refine(Fz, b, tol=1e-12, max_iter=10)
    assert hist[-1] <= 1e-12 and len(hist) <= 8
    assert np.linalg.norm(Zh @ x - b) / np.linalg.norm(b) < 1e-11


# ---------------------------------------------- planted mistakes (CPU) ----


def test_planted_mistakes_are_caught(monkeypatch):
    """A plausible mistake in the oracle must fail one of the pins above."""
    Hm = h2_problem(12, 64, 1e-6)
    Zh = h2_dense(12, 64, 1e-6)
    b = inputs.rhs_gaussian(Hm.tree.N, 1, 2)[:, 0]
    xe = np.linalg.solve(Zh, b)

    def err_exact():
        x = factor.solve(factor.factorize(Hm, 0.0), b)
        return np.linalg.norm(x - xe) / np.linalg.norm(xe)

    import scipy.linalg as sla
    # (a) transposed operand in the L panel Z_ci' U^{-1}
    monkeypatch.setattr(factor, "_x_uinv", lambda X, LU: sla.solve_triangular(LU, X.T, lower=False).T)
    assert err_exact() > 1e-6
    monkeypatch.undo()
    # (b) dropped row permutation in L^{-1} P
    monkeypatch.setattr(factor, "_linv_p", lambda LU, piv, X: sla.solve_triangular(LU, X, lower=True, unit_diagonal=True))
    assert err_exact() > 1e-6
    monkeypatch.undo()
    # (c) conjugated self term (wrong sign of the imaginary part)
    st = kernel.self_term
    monkeypatch.setattr(kernel, "self_term", lambda k, h: np.conj(st(k, h)))
    with pytest.raises(AssertionError):
        test_self_term_quadrature()
    monkeypatch.undo()
    assert err_exact() < 1e-11
    # (d) block LDL^T with the conjugate transpose where Z^T = Z asks for the
    # plain transpose
    monkeypatch.setattr(factor, "_transpose", lambda X: X.conj().T)
    x = factor.solve(factor.factorize(Hm, 0.0, symmetric=True), b)
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) > 1e-6
    monkeypatch.undo()


# ------------------------------------------- derivative in the contrast ----


def test_adjoint_lu_solve_against_lapack():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    c = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    LU, piv = dense.lu(A)
    y = dense.lu_solve_adjoint(LU, piv, c)
    assert np.linalg.norm(y - np.linalg.solve(A.conj().T, c)) <= 1e-12 * np.linalg.norm(y)


def test_grad_one_unknown_closed_form():
    # N = 1: A = 1 + s kappa chi, x = b / A, L = |x|^2 (g = 2 x):
    # dL/dchi = -2 |b|^2 Re(conj(A) s kappa) / |A|^4
    from oracle import adjoint
    kappa = kernel.self_term(K, H)
    for s in (1.0, -1.0):
        for chi in (0.5, 1.75, 3.0):
            b = 0.3 - 1.1j
            A = 1.0 + s * kappa * chi
            x = b / A
            g = 2.0 * x
            mu = g / np.conj(A)
            got = adjoint.grad_reduced(np.array([chi]), np.array([x]), np.array([mu]), np.array([g]))[0]
            ref = -2.0 * abs(b) ** 2 * np.real(np.conj(A) * s * kappa) / abs(A) ** 4
            assert abs(got - ref) <= 1e-12 * abs(ref)


def _grad_problem(n=4, seed=4):
    from oracle import adjoint
    pts = inputs.grid_points(n, H)
    N = len(pts)
    chi = inputs.chi_random_cells(N, seed)
    b = inputs.rhs_plane_wave(pts, K)
    radius = 2.0 * (math.sqrt(3.0) / 2.0) * n * H
    probes = inputs.fibonacci_sphere(64, pts.mean(axis=0), radius)
    G = adjoint.probe_matrix(probes, pts, K, H)
    return pts, chi, b, G


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_probe_gradient_forms_match_finite_differences(sign):
    # reduced 2 Re(x conj(lambda)) / chi == general 2 Re(x conj(w - s K^H lambda))
    # == central differences of dense solves (step 1e-6, error ~1e-10 relative)
    from oracle import adjoint
    pts, chi, b, G = _grad_problem()
    A = kernel.dense_A(pts, chi, K, H, sign)
    Kd = adjoint.dense_K(pts, K, H)
    _, _, red, gen = adjoint.probe_gradient(A, Kd, G, chi, b, sign)
    cells = [0, 7, 21, 63]
    fd = adjoint.probe_fd(pts, chi, K, H, b, G, cells, 1e-6, sign)
    scale = np.max(np.abs(red))
    assert np.max(np.abs(red - gen)) <= 1e-12 * scale
    assert np.max(np.abs(red[cells] - fd)) <= 1e-7 * scale


def test_solve_gradient_with_incoming_g_matches_finite_differences():
    # the solve-only derivative used by the autograd node: L = sum |W x|^2 for a
    # fixed complex W (no chi outside the solve), g = 2 W^H W x
    from oracle import adjoint
    pts, chi, b, G = _grad_problem()
    A = kernel.dense_A(pts, chi, K, H)
    Kd = adjoint.dense_K(pts, K, H)
    x = dense.solve(A, b)
    g = 2.0 * (G.conj().T @ (G @ x))
    mu = dense.solve(A.conj().T, g)
    red = adjoint.grad_reduced(chi, x, mu, g)
    gen = adjoint.grad_general(Kd, 1.0, x, mu)
    cells = [3, 30, 60]
    fd = []
    for i in cells:
        v = []
        for d in (1e-6, -1e-6):
            c = chi.copy()
            c[i] += d
            xi = dense.solve(kernel.dense_A(pts, c, K, H), b)
            v.append(np.sum(np.abs(G @ xi) ** 2))
        fd.append((v[0] - v[1]) / 2e-6)
    scale = np.max(np.abs(red))
    assert np.max(np.abs(red - gen)) <= 1e-12 * scale
    assert np.max(np.abs(red[cells] - np.array(fd))) <= 1e-7 * scale
    # planted mistake: dropping g (using the probe form without the direct
    # term) is visibly wrong
    bad = adjoint.grad_reduced(chi, x, mu)
    assert np.max(np.abs(bad[cells] - np.array(fd))) > 1e-3 * scale
