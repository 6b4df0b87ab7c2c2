"""Block LDL^T form of the elimination (h2_opts.ldlt = 1; the default 2 takes
it for FP64 factorizations of a complex-symmetric matrix) on the GPU against
the oracle's block LDL^T (factor.factorize(..., symmetric=True)) on the same
H^2 matrices (h2_load), and against the block LU form (ldlt = 0).

Tolerances, as for the LU form:
  * eps_fill = 0: the factorization is exact, 1e-10 against a dense solve;
  * eps_fill = eps: 10 eps relative to the oracle's solution; per-cluster kept
    ranks within +-1 (at a threshold tie one side may keep a direction the
    other drops);
  * refined solutions: the exact H^2 solution to 1e-11 (FP64 factors) or the
    requested tolerance (mixed).
"""
import numpy as np
import pytest

from oracle import factor
from paper_1703_06155_gb300 import inputs

from _h2io import from_tree, oracle_to_rep, to_tree
from _problems import H, K, h2_dense, h2_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-6


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1703_06155_gb300 import lib
    lib()
    return torch.device("cuda:0")


def load(Hm, **kw):
    from paper_1703_06155_gb300 import H2
    return H2.load(oracle_to_rep(Hm), **kw)


def test_ldlt_exact(dev):
    Hm = h2_problem(12, 64, EPS)
    Zd = h2_dense(12, 64, EPS)
    # the default takes block LDL^T for FP64 and block LU for the mixed bulk
    A = load(Hm)
    A.factorize(EPS, "mixed")
    assert A.stats()["ldlt"] == 0
    A.factorize(0.0, "fp64")
    assert A.stats()["ldlt"] == 1
    b = inputs.rhs_gaussian(Hm.tree.N, 2, 11)
    xe = from_tree(Hm, np.linalg.solve(Zd, to_tree(Hm, b)))
    bt = torch.from_numpy(b).to(dev)
    x = A.solve(bt).cpu().numpy()
    assert rel(x, xe) < 1e-10
    xa = A.solve(bt, adjoint=True).cpu().numpy()
    xae = from_tree(Hm, np.linalg.solve(Zd.conj().T, to_tree(Hm, b)))
    assert rel(xa, xae) < 1e-10
    A.invert()
    xi = A.solve(bt, use_inverse=True).cpu().numpy()
    assert rel(xi, x) < 1e-12
    A.close()


@pytest.mark.parametrize("n", [12, 16])
def test_ldlt_fp64_parity(dev, n):
    Hm = h2_problem(n, 64, EPS)
    Fz = factor.factorize(Hm, EPS, "colored", symmetric=True)
    b = inputs.rhs_gaussian(Hm.tree.N, 1, 0)[:, 0]
    x_orc = from_tree(Hm, factor.solve(Fz, to_tree(Hm, b)))
    A = load(Hm, ldlt=1)
    A.factorize(EPS, "fp64")
    x = A.solve(b)
    assert rel(x, x_orc) <= 10 * EPS, rel(x, x_orc)
    worst = 0
    for li, lev in enumerate(Fz.levels):
        _, kt = A.level_ranks(Hm.L - li)
        worst = max(worst, int(np.abs(kt.astype(int) - lev.kt.astype(int)).max()))
    assert worst <= 1, worst
    Zd = h2_dense(n, 64, EPS)
    xr = A.solve(b, refine=True, tol=1e-13, max_iter=10)
    xe = from_tree(Hm, np.linalg.solve(Zd, to_tree(Hm, b)))
    assert rel(xr, xe) < 1e-11
    # adjoint against the oracle's (conj Z^-1 conj)
    xa = A.solve(b, adjoint=True)
    xa_orc = from_tree(Hm, factor.solve_adjoint(Fz, to_tree(Hm, b)))
    assert rel(xa, xa_orc) <= 10 * EPS
    A.close()


def test_ldlt_mixed_refinement_and_memory(dev):
    # the same matrix factorized in both forms (fresh contexts, so the
    # grow-only arenas do not mix): same refined solution, the near-field
    # factor blocks about halved
    Hm = h2_problem(16, 64, EPS)
    b = inputs.rhs_gaussian(Hm.tree.N, 3, 2)
    out = {}
    for ld in (0, 1):
        A = load(Hm, ldlt=ld)
        A.factorize(EPS, "mixed")
        x = A.solve(b, refine=True, tol=1e-10, max_iter=30)
        st = A.stats()
        out[ld] = (x, A.last_solve["resid"], st["mem"]["near_blocks"], st["ldlt"])
        A.close()
    assert out[0][1] <= 1e-10 and out[1][1] <= 1e-10
    assert out[0][3] == 0 and out[1][3] == 1
    assert rel(out[1][0], out[0][0]) < 1e-8
    ratio = out[1][2] / out[0][2]
    print("near-field factor blocks, LDL^T / LU: %.3f" % ratio)
    assert 0.45 <= ratio <= 0.65, ratio


def test_ldlt_batch_and_form_checks(dev):
    from paper_1703_06155_gb300 import H2Error, factorize_batch, solve_batch
    H12, H16 = h2_problem(12, 64, EPS), h2_problem(16, 64, EPS)
    A, B = load(H12, ldlt=1), load(H16, ldlt=1)
    factorize_batch([A, B], EPS, "fp64")
    b12 = inputs.rhs_gaussian(H12.tree.N, 2, 3)
    b16 = inputs.rhs_gaussian(H16.tree.N, 2, 4)
    bs = [torch.from_numpy(b12).to(dev), torch.from_numpy(b16).to(dev)]
    xs, _ = solve_batch([A, B], bs)
    for Hm, bb, x in ((H12, b12, xs[0]), (H16, b16, xs[1])):
        Fz = factor.factorize(Hm, EPS, "colored", symmetric=True)
        assert rel(x.cpu().numpy(), from_tree(Hm, factor.solve(Fz, to_tree(Hm, bb)))) <= 10 * EPS
    xa, _ = solve_batch([A, B], bs, adjoint=True)
    assert rel(xa[0].cpu().numpy(), A.solve(b12, adjoint=True)) < 1e-12
    # a batch whose instances do not all ask for LDL^T runs in the LU form
    C = load(H12, ldlt=0)
    factorize_batch([A, C], EPS, "fp64")
    assert A.stats()["ldlt"] == 0 and C.stats()["ldlt"] == 0
    # contexts factorized in different forms are not solved together
    B.factorize(EPS, "fp64")
    assert B.stats()["ldlt"] == 1
    with pytest.raises(H2Error):
        solve_batch([A, B], bs)
    # a matrix that is not symmetric is factorized in the LU form
    rep = oracle_to_rep(H12)
    pairs = H12.part.inad[H12.L]
    sizes = np.asarray(H12.tree.size[H12.L])
    q = next(u for u, (s, t) in enumerate(pairs) if s != t)
    off = int(sum(sizes[s] * sizes[t] for s, t in pairs[:q]))
    rep["D"] = rep["D"].copy()
    rep["D"][off] += 1e-3
    from paper_1703_06155_gb300 import H2
    D = H2.load(rep, ldlt=1)
    assert D.stats()["symmetric"] == 0
    D.factorize(0.0, "fp64")
    assert D.stats()["ldlt"] == 0
    x = D.solve(b12)
    assert rel(D.matvec(x), b12) < 1e-10
    for c in (A, B, C, D):
        c.close()


def test_ldlt_benchmark_grid32(dev):
    # the benchmark workload (32^3, library construction, mixed precision,
    # 16 right-hand sides) in both forms: refined solutions to 1e-6 that agree
    # to 1e-5, per-level largest ranks within a few directions (the Step-0
    # decisions see the same Schur complements up to rounding), the LDL^T
    # near-field factors about half
    from paper_1703_06155_gb300 import H2
    n = 32
    pts = inputs.grid_points(n, H)
    N = len(pts)
    b = torch.from_numpy(inputs.rhs_gaussian(N, 16, 0)).to(dev)
    out = {}
    for ld in (0, 1):
        A = H2.build(pts, K, H, 3.0, EPS, ldlt=ld)
        A.factorize(EPS, "mixed")  # warm-up of the arenas
        A.factorize(EPS, "mixed")
        st = A.stats()
        x = A.solve(b, refine=True, tol=1e-6, max_iter=30).cpu().numpy()
        out[ld] = (x, A.last_solve["resid"], st["t_factor_ms"], st["mem"]["near_blocks"],
                   [lv["kt_max"] for lv in st["levels"]])
        A.close()
    print("grid32 mixed factorization: LU %.1f ms, LDL^T %.1f ms; near-field factors %.2f / %.2f GB; "
          "kt_max %s / %s" % (out[0][2], out[1][2], out[0][3] / 1e9, out[1][3] / 1e9, out[0][4], out[1][4]))
    assert out[0][1] <= 1e-6 and out[1][1] <= 1e-6
    assert rel(out[1][0], out[0][0]) <= 1e-5
    assert all(abs(a - c) <= 3 for a, c in zip(out[0][4], out[1][4]))
    assert out[1][3] <= 0.65 * out[0][3]
