"""GPU path vs the CPU oracle on the same seeded H^2 matrices (C ABI via the
ctypes binding).  The oracle's H^2 representation is handed to h2_load, so
both sides factorize exactly the same matrix.

Tolerances (floating point, complex128 unless stated):
  * matvec: 1e-13 relative (same arithmetic, different summation order);
  * eps_fill = 0: the factorization is an exact block LU of Z_H2, so the
    solution matches a dense solve to 1e-10;
  * eps_fill = eps: GPU and oracle keep fill-in directions by the same rule,
    but at a threshold tie a direction can be kept by one side only (ranks
    +-1), which perturbs the solution by O(eps).  Bound: 10 eps relative to
    the oracle's solution, as long as the oracle's own residual is <= eps.
"""
import numpy as np
import pytest

from oracle import factor
from oracle import h2 as oh2
from paper_1703_06155_gb300 import inputs

from _h2io import from_tree, oracle_to_rep, to_tree
from _problems import factorization, h2_dense, h2_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1703_06155_gb300 import lib
    lib()
    return torch.device("cuda:0")


def gpu_ctx(H, **kw):
    from paper_1703_06155_gb300 import H2
    return H2.load(oracle_to_rep(H), **kw)


def oracle_solve(Fz, b_global, adjoint=False):
    H = Fz.H
    if adjoint:
        return from_tree(H, factor.solve_adjoint(Fz, to_tree(H, b_global)))
    return from_tree(H, factor.solve(Fz, to_tree(H, b_global)))


@pytest.mark.parametrize("n", [12, 16])
def test_matvec_parity(dev, n):
    H = h2_problem(n, 64, 1e-6)
    A = gpu_ctx(H)
    x = inputs.rhs_gaussian(H.tree.N, 3, 5)
    y_ref = from_tree(H, oh2.matvec(H, to_tree(H, x)))
    y = A.matvec(torch.from_numpy(x).to(dev)).cpu().numpy()
    assert rel(y, y_ref) < 1e-13
    yh = A.matvec(x)  # host buffers
    assert rel(yh, y_ref) < 1e-13
    # adjoint product against the dense conjugate transpose
    Zd = h2_dense(n, 64, 1e-6)
    ya = A.matvec(x, adjoint=True)
    ya_ref = from_tree(H, Zd.conj().T @ to_tree(H, x))
    assert rel(ya, ya_ref) < 1e-13


@pytest.mark.parametrize("ordering,apply_path", [("colored", 1), ("natural", 1), ("colored", 2)])
def test_exact_block_lu(dev, ordering, apply_path):
    H = h2_problem(12, 64, 1e-6)
    A = gpu_ctx(H, ordering=ordering, apply_path=apply_path)
    A.factorize(0.0, "fp64")
    Zd = h2_dense(12, 64, 1e-6)
    b = inputs.rhs_gaussian(H.tree.N, 2, 11)
    xe = from_tree(H, np.linalg.solve(Zd, to_tree(H, b)))
    x = A.solve(torch.from_numpy(b).to(dev)).cpu().numpy()
    assert rel(x, xe) < 1e-10
    xa = A.solve(b, adjoint=True)
    xae = from_tree(H, np.linalg.solve(Zd.conj().T, to_tree(H, b)))
    assert rel(xa, xae) < 1e-10


@pytest.mark.parametrize("n,eps,apply_path", [(12, 1e-6, 0), (16, 1e-6, 0), (12, 1e-4, 0), (16, 1e-6, 2)])
def test_fp64_parity(dev, n, eps, apply_path):
    H = h2_problem(n, 64, eps)
    Fz = factorization(n, 64, eps, eps, "colored")
    A = gpu_ctx(H, apply_path=apply_path)
    A.factorize(eps, "fp64")
    b = inputs.rhs_gaussian(H.tree.N, 1, 0)[:, 0]
    x_orc = oracle_solve(Fz, b)
    Zd = h2_dense(n, 64, eps)
    res_orc = np.linalg.norm(Zd @ to_tree(H, x_orc) - to_tree(H, b)) / np.linalg.norm(b)
    x = A.solve(b)
    res_gpu = np.linalg.norm(Zd @ to_tree(H, x) - to_tree(H, b)) / np.linalg.norm(b)
    assert res_orc <= eps and res_gpu <= 10 * eps, (res_orc, res_gpu)
    assert rel(x, x_orc) <= 10 * eps, rel(x, x_orc)
    # ranks: per level, the largest kept rank agrees within a few directions
    st = A.stats()
    for lev, olev in zip(st["levels"], Fz.levels):
        assert abs(lev["kt_max"] - int(olev.kt.max())) <= 2, (lev, olev.kt.max())
    # after refinement both solutions agree with the exact H^2 solution
    xr = A.solve(b, refine=True, tol=1e-13, max_iter=10)
    xe = from_tree(H, np.linalg.solve(Zd, to_tree(H, b)))
    assert rel(xr, xe) < 1e-11


def test_inverse_and_adjoint(dev):
    eps = 1e-6
    H = h2_problem(12, 64, eps)
    Fz = factorization(12, 64, eps, eps, "colored")
    A = gpu_ctx(H)
    A.factorize(eps, "fp64")
    b = inputs.rhs_gaussian(H.tree.N, 4, 9)
    bt = torch.from_numpy(b).to(dev)
    x = A.solve(bt).cpu().numpy()
    A.invert()
    xi = A.solve(bt, use_inverse=True).cpu().numpy()
    assert rel(xi, x) < 1e-12
    xa = A.solve(bt, adjoint=True).cpu().numpy()
    xa_orc = oracle_solve(Fz, b, adjoint=True)
    assert rel(xa, xa_orc) <= 10 * eps
    # <A^H y, x> = <y, A x> with the GPU adjoint solve and matvec
    y = inputs.rhs_gaussian(H.tree.N, 1, 3)[:, 0]
    u = A.solve(y, adjoint=True)
    v = b[:, 0]
    lhs = np.vdot(u, A.matvec(A.solve(v)))
    rhs = np.vdot(A.matvec(u, adjoint=True), A.solve(v))
    assert abs(lhs - rhs) / abs(lhs) < 1e-10


def test_mixed_precision_refinement(dev):
    eps = 1e-6
    H = h2_problem(12, 64, eps)
    A = gpu_ctx(H)
    A.factorize(eps, "mixed")
    b = inputs.rhs_gaussian(H.tree.N, 2, 1)
    Zd = h2_dense(12, 64, eps)
    x = A.solve(b, refine=True, tol=1e-10, max_iter=30)
    assert A.last_solve["resid"] <= 1e-10
    xe = from_tree(H, np.linalg.solve(Zd, to_tree(H, b)))
    assert rel(x, xe) < 1e-8


def test_singular_pivot_reports_status(dev):
    # a leaf diagonal block that is exactly zero where the partial LU pivots;
    # the natural order eliminates cluster 0 first, before any Schur update
    # could fill its diagonal block
    from paper_1703_06155_gb300 import H2Error
    H = h2_problem(12, 64, 1e-6)
    rep = oracle_to_rep(H)
    n0 = int(rep["leaf_size"][0])
    rep["D"] = rep["D"].copy()
    rep["D"][: n0 * n0] = 0  # first near block is (0, 0)
    A = gpu_ctx_rep(rep, ordering="natural")
    with pytest.raises(H2Error) as ei:
        A.factorize(1e-6, "fp64")
    assert ei.value.status == -3


def gpu_ctx_rep(rep, **kw):
    from paper_1703_06155_gb300 import H2
    return H2.load(rep, **kw)


def test_solve_graph_replay(dev):
    # h2_opts.solve_graph: 1st solve runs normally, 2nd is captured, later ones
    # replay the CUDA graph; all must equal the plain launches bit for bit, and
    # a refactorization must retire the graph
    eps = 1e-6
    H = h2_problem(12, 64, eps)
    A0 = gpu_ctx(H)
    A1 = gpu_ctx(H, solve_graph=1)
    s = torch.cuda.Stream()
    b = torch.from_numpy(inputs.rhs_gaussian(H.tree.N, 3, 17)).to(dev)
    for prec in ("mixed", "fp64"):
        A0.factorize(eps, prec)
        A1.factorize(eps, prec)
        with torch.cuda.stream(s):
            ref = A0.solve(b, stream=s)
            refa = A0.solve(b, adjoint=True, stream=s)
            for _ in range(4):
                x = A1.solve(b, stream=s)
                xa = A1.solve(b, adjoint=True, stream=s)
                assert torch.equal(x, ref) and torch.equal(xa, refa)
            xr = A1.solve(b, refine=True, tol=1e-12, max_iter=20, stream=s)
        s.synchronize()
        Zd = h2_dense(12, 64, eps)
        xe = from_tree(H, np.linalg.solve(Zd, to_tree(H, b.cpu().numpy())))
        assert rel(xr.cpu().numpy(), xe) < 1e-10


def test_autotune_keeps_results(dev):
    # the tuner only picks among equivalent execution settings: the solution
    # stays the exact-block-LU one at eps = 0 for every setting it leaves
    from paper_1703_06155_gb300.autotune import autotune
    H = h2_problem(12, 64, 1e-6)
    A = gpu_ctx(H)
    b = torch.from_numpy(inputs.rhs_gaussian(H.tree.N, 2, 3)).to(dev)
    best, log = autotune(A, b, 0.0, "fp64", tol=1e-12, repeats=1,
                         space={"tile_policy": [0, 1], "cluster_max": [16, 4], "apply_path": [2, 1]})
    assert set(best) == {"tile_policy", "cluster_max", "apply_path"} and len(log) >= 4
    A.factorize(0.0, "fp64")
    Zd = h2_dense(12, 64, 1e-6)
    x = A.solve(b).cpu().numpy()
    xe = from_tree(H, np.linalg.solve(Zd, to_tree(H, b.cpu().numpy())))
    assert rel(x, xe) < 1e-10


@pytest.mark.parametrize("tc", [2, 0])
def test_split_k_tiles_match_direct_tiles(dev, tc):
    # a split-K target far above the GPU's CTA count cuts the long products of
    # every GEMM launch into K chunks whose partial tiles (tensor-core or FMA
    # kernels) are summed by the reduction pass: FP32-close to the default plan,
    # and both refine to the exact H^2 solution
    eps = 1e-6
    n = 16
    H = h2_problem(n, 64, eps)
    A1 = gpu_ctx(H, tensor_cores=tc, split_target=20000)
    A0 = gpu_ctx(H, tensor_cores=tc)
    A1.factorize(eps, "mixed")
    A0.factorize(eps, "mixed")
    b = torch.from_numpy(inputs.rhs_gaussian(H.tree.N, 2, 31)).to(dev)
    x1, x0 = A1.solve(b).cpu().numpy(), A0.solve(b).cpu().numpy()
    assert rel(x1, x0) < 1e-4
    Zd = h2_dense(n, 64, eps)
    xe = from_tree(H, np.linalg.solve(Zd, to_tree(H, b.cpu().numpy())))
    xr = A1.solve(b, refine=True, tol=1e-12, max_iter=30).cpu().numpy()
    assert rel(xr, xe) < 1e-10


def test_gram_emulation_matches_fp64_grams(dev):
    # Step-0 Grams of complex64 operands as exact products summed in
    # double-float on the FP32 pipe (flushed to FP64 every 8 terms) or with
    # FP64 FMAs: the same Step-0 ranks on every level, FP32-close
    # factorizations, and both refine to the exact H^2 solution
    eps = 1e-6
    n = 16
    H = h2_problem(n, 64, eps)
    A1 = gpu_ctx(H, gram_emulation=1)
    A0 = gpu_ctx(H, gram_emulation=0)
    A1.factorize(eps, "mixed")
    A0.factorize(eps, "mixed")
    e1 = [lv["eliminated"] for lv in A1.stats()["levels"]]
    e0 = [lv["eliminated"] for lv in A0.stats()["levels"]]
    assert e1 == e0
    b = torch.from_numpy(inputs.rhs_gaussian(H.tree.N, 2, 29)).to(dev)
    x1, x0 = A1.solve(b).cpu().numpy(), A0.solve(b).cpu().numpy()
    assert rel(x1, x0) < 1e-4
    Zd = h2_dense(n, 64, eps)
    xe = from_tree(H, np.linalg.solve(Zd, to_tree(H, b.cpu().numpy())))
    xr = A1.solve(b, refine=True, tol=1e-12, max_iter=30).cpu().numpy()
    assert rel(xr, xe) < 1e-10


@pytest.mark.parametrize("tc", [1, 2])
def test_tensor_core_bulk_matches_fma_bulk(dev, tc):
    # the complex64 bulk on the tensor cores (3xTF32: warp-level MMAs, or
    # tcgen05 MMAs accumulating in tensor memory) and on the FP32 FMA pipe
    # give FP32-close factorizations; both refine to the exact H^2 solution
    eps = 1e-6
    n = 16
    H = h2_problem(n, 64, eps)
    A1 = gpu_ctx(H, tensor_cores=tc)
    A0 = gpu_ctx(H, tensor_cores=0)
    A1.factorize(eps, "mixed")
    A0.factorize(eps, "mixed")
    b = torch.from_numpy(inputs.rhs_gaussian(H.tree.N, 2, 23)).to(dev)
    x1, x0 = A1.solve(b).cpu().numpy(), A0.solve(b).cpu().numpy()
    assert rel(x1, x0) < 1e-4
    Zd = h2_dense(n, 64, eps)
    xe = from_tree(H, np.linalg.solve(Zd, to_tree(H, b.cpu().numpy())))
    assert rel(x1, xe) < 1e-4
    xr = A1.solve(b, refine=True, tol=1e-12, max_iter=30).cpu().numpy()
    assert rel(xr, xe) < 1e-10


@pytest.mark.parametrize("N", [1, 7, 65, 129])
def test_degenerate_sizes_solve(dev, N):
    # one point, fewer points than a leaf (the whole matrix is the final block),
    # one point past a leaf and a ragged two-level tree: GPU build (library
    # construction), FP64 and mixed factorizations, solves against the exact
    # dense solution of the same points
    from oracle import kernel
    from paper_1703_06155_gb300 import H2
    pts = np.ascontiguousarray(inputs.grid_points(6, 1.0 / 16.0)[:N])
    chi = inputs.chi_uniform(N, 3.0)
    eps = 1e-8
    A = H2.build(pts, 2 * np.pi, 1.0 / 16.0, chi, eps)
    idx = np.arange(N)
    Z = kernel.entries(pts, chi, idx, idx, 2 * np.pi, 1.0 / 16.0)
    b = inputs.rhs_gaussian(N, 2, 37)
    xe = np.linalg.solve(Z, b)
    A.factorize(eps, "fp64")
    x = A.solve(torch.from_numpy(b).to(dev)).cpu().numpy()
    assert rel(x, xe) < 1e-6
    A.factorize(eps, "mixed")
    xm = A.solve(torch.from_numpy(b).to(dev), refine=True, tol=1e-12, max_iter=30).cpu().numpy()
    assert rel(xm, xe) < 1e-6
    A.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_refactorization_is_bitwise_repeatable(dev, prec):
    # the factorization has no order-dependent arithmetic (no atomics on
    # values, fixed split-K reduction order): refactorizing one context, and
    # factorizing a fresh one, must reproduce the solution bit for bit.  The
    # scratch and factor arenas of a context are reused, so a kernel that read
    # memory before writing it, or a missing barrier, would show up here as
    # occasional differences
    eps = 1e-6
    H = h2_problem(16, 64, eps)
    b = torch.from_numpy(inputs.rhs_gaussian(H.tree.N, 2, 29)).to(dev)
    A = gpu_ctx(H)
    xs = []
    for _ in range(8):
        A.factorize(eps, prec)
        xs.append(A.solve(b).cpu().numpy())
    B = gpu_ctx(H)
    B.factorize(eps, prec)
    xs.append(B.solve(b).cpu().numpy())
    diffs = [float(np.abs(x - xs[0]).max()) for x in xs[1:]]
    print("%s refactorizations: largest difference to the first %s" % (prec, diffs))
    assert max(diffs) == 0.0
    A.close()
    B.close()
