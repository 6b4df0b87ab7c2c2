"""Batched instances (h2_factorize_batch / h2_solve_batch): several
independent H^2 matrices of different depth factorized and solved in shared
launches, checked per instance against dense solves (eps_fill = 0: exact block
LU), against the CPU oracle (eps_fill = eps: 10 eps, as for one instance) and
against the same instances factorized one by one."""
import numpy as np
import pytest

from oracle import factor
from paper_1703_06155_gb300 import inputs

from _h2io import from_tree, oracle_to_rep, to_tree
from _problems import factorization, h2_dense, h2_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (grid, percell seed): depths L = 5, 6, 5; uniform and per-cell contrast
CASES = [(12, None), (16, None), (12, 4)]
EPS = 1e-6


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1703_06155_gb300 import lib
    lib()
    return torch.device("cuda:0")


def contexts():
    from paper_1703_06155_gb300 import H2
    out = []
    for n, seed in CASES:
        H = h2_problem(n, 64, EPS, percell_seed=seed)
        chi = inputs.chi_random_cells(H.tree.N, seed) if seed is not None else None
        out.append(H2.load(oracle_to_rep(H, dscale=None if chi is None else np.sqrt(chi))))
    return out


def rhs(nrhs, seed):
    return [inputs.rhs_gaussian(h2_problem(n, 64, EPS, percell_seed=s).tree.N, nrhs, seed + i)
            for i, (n, s) in enumerate(CASES)]


def dense_solve(q, b, adjoint=False):
    n, seed = CASES[q]
    H = h2_problem(n, 64, EPS, percell_seed=seed)
    Zd = h2_dense(n, 64, EPS, percell_seed=seed)
    sc = np.ones(H.tree.N) if seed is None else np.sqrt(inputs.chi_random_cells(H.tree.N, seed))
    # A = S^{-1} Z S in global order; Z (S x) = S b; adjoint: Z^H (S^{-1} x) = S^{-1} b
    s_t = to_tree(H, sc)
    if not adjoint:
        y = np.linalg.solve(Zd, s_t[:, None] * to_tree(H, b))
        return from_tree(H, y / s_t[:, None])
    y = np.linalg.solve(Zd.conj().T, to_tree(H, b) / s_t[:, None])
    return from_tree(H, y * s_t[:, None])


def test_batch_exact_block_lu(dev):
    from paper_1703_06155_gb300 import factorize_batch, solve_batch
    cs = contexts()
    factorize_batch(cs, 0.0, "fp64")
    bs = rhs(3, 21)
    xs, _ = solve_batch(cs, [torch.from_numpy(b).to(dev) for b in bs])
    for q, (x, b) in enumerate(zip(xs, bs)):
        assert rel(x.cpu().numpy(), dense_solve(q, b)) < 1e-10, q
    xa, _ = solve_batch(cs, [torch.from_numpy(b).to(dev) for b in bs], adjoint=True)
    for q, (x, b) in enumerate(zip(xa, bs)):
        assert rel(x.cpu().numpy(), dense_solve(q, b, adjoint=True)) < 1e-10, q


def test_batch_fp64_matches_oracle_and_single(dev):
    from paper_1703_06155_gb300 import factorize_batch, solve_batch
    cs = contexts()
    factorize_batch(cs, EPS, "fp64")
    single = contexts()
    for c in single:
        c.factorize(EPS, "fp64")
    bs = rhs(1, 5)
    xs, _ = solve_batch(cs, [torch.from_numpy(b).to(dev) for b in bs])
    for q, ((n, seed), x, b) in enumerate(zip(CASES, xs, bs)):
        x = x.cpu().numpy()
        Fz = factorization(n, 64, EPS, EPS, "colored", percell_seed=seed)
        H = Fz.H
        sc = np.ones(H.tree.N) if seed is None else np.sqrt(inputs.chi_random_cells(H.tree.N, seed))
        s_t = to_tree(H, sc)
        x_orc = from_tree(H, factor.solve(Fz, s_t[:, None] * to_tree(H, b)) / s_t[:, None])
        assert rel(x, x_orc) <= 10 * EPS, (q, rel(x, x_orc))
        x1 = single[q].solve(torch.from_numpy(b).to(dev)).cpu().numpy()
        assert rel(x, x1) <= 10 * EPS, (q, rel(x, x1))


def test_batch_mixed_refinement(dev):
    from paper_1703_06155_gb300 import factorize_batch, solve_batch
    cs = contexts()
    factorize_batch(cs, EPS, "mixed")
    bs = rhs(4, 9)
    xs, info = solve_batch(cs, [torch.from_numpy(b).to(dev) for b in bs], refine=True, tol=1e-10, max_iter=30)
    assert info["resid"] <= 1e-10
    for q, (x, b) in enumerate(zip(xs, bs)):
        assert rel(x.cpu().numpy(), dense_solve(q, b)) < 1e-8, q


def test_many_instances_share_launches(dev):
    # 24 copies of one 16^3 problem in one batch: a Step-0 launch then holds
    # about a hundred eigen-problems, so the per-problem clusters get small
    # and the one-sided Jacobi's column blocks long (they must stay within
    # the kernel's block limit); every instance must match the same problem
    # factorized alone, to FP32 closeness before refinement and to 1e-10 after
    from paper_1703_06155_gb300 import H2, factorize_batch, solve_batch
    H = h2_problem(16, 64, EPS)
    rep = oracle_to_rep(H)
    cs = [H2.load(rep) for _ in range(24)]
    factorize_batch(cs, EPS, "mixed")
    one = H2.load(rep)
    one.factorize(EPS, "mixed")
    b = inputs.rhs_gaussian(H.tree.N, 2, 41)
    bt = torch.from_numpy(b).to(dev)
    x1 = one.solve(bt).cpu().numpy()
    xs, _ = solve_batch(cs, [bt] * len(cs))
    worst = max(rel(x.cpu().numpy(), x1) for x in xs)
    xr, _ = solve_batch(cs, [bt] * len(cs), refine=True, tol=1e-10, max_iter=30)
    xr1 = one.solve(bt, refine=True, tol=1e-10, max_iter=30).cpu().numpy()
    worst_r = max(rel(x.cpu().numpy(), xr1) for x in xr)
    print("24 instances: unrefined vs alone %.1e, refined vs alone %.1e" % (worst, worst_r))
    assert worst < 1e-4 and worst_r < 1e-9
    for c in cs + [one]:
        c.close()
