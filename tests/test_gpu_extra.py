"""GPU checks of the construction, the explicit inverse, the failure statuses
and the contrast update, each against something independent of the CUDA path:

* h2_build on the GPU (far-field Grams in k_kgram) against the dense kernel
  matrix (10 eps_build) and against the same build done on the host;
* H2_USE_INVERSE solves (eq. 35) against the oracle's explicit inverse and
  against a dense solve;
* H2_ENOMEM from the arena cap, H2_ENOCONV from a refinement that cannot
  reach its tolerance, and a context that stays usable after both;
* h2_set_chi against the dense rescaled matrix, and the autograd node taking
  a gradient step in chi on one context against a dense solve at the new chi.
"""
import numpy as np
import pytest

from oracle import adjoint, factor, kernel
from oracle import h2 as oh2
from paper_1703_06155_gb300 import inputs

from _h2io import dense_from_rep, from_tree, oracle_to_rep, to_tree
from _problems import H, K, factorization, h2_dense, h2_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


@pytest.mark.parametrize("n", [12, 16])
def test_gpu_build_matches_dense_and_host_build(dev, n):
    from paper_1703_06155_gb300 import H2
    eps = 1e-6
    pts = inputs.grid_points(n, H)
    N = len(pts)
    chi = inputs.chi_random_cells(N, 4)
    A = H2.build(pts, K, H, chi, eps)  # GPU far-field Grams
    B = H2.build(pts, K, H, chi, eps, host_only=1)
    ra, rb = A.export(), B.export()
    assert np.array_equal(ra["perm"], rb["perm"])
    Za, _ = dense_from_rep(ra)
    Zb, _ = dense_from_rep(rb)
    idx = ra["perm"]
    Zex = kernel.entries(pts, chi, idx, idx, K, H)
    ea, eb = rel(Za, Zex), rel(Zb, Zex)
    print("grid%d build: GPU %.2e, host %.2e of ||Z||_F; ranks equal on %.1f %% of the clusters" % (
        n, ea, eb, 100.0 * np.mean(ra["rank"] == rb["rank"])))
    assert ea < 10 * eps and eb < 10 * eps
    assert rel(Za, Zb) < 10 * eps
    # the two Gram orders differ only in rounding: pivot decisions at ties aside,
    # the same skeleton ranks
    assert np.mean(ra["rank"] == rb["rank"]) >= 0.95
    A.close()
    B.close()


def test_inverse_matches_oracle_inverse_and_dense(dev):
    eps = 1e-6
    Hm = h2_problem(12, 64, eps)
    Fz = factorization(12, 64, eps, eps, "colored")
    inv = factor.invert(Fz)
    from paper_1703_06155_gb300 import H2
    A = H2.load(oracle_to_rep(Hm))
    A.factorize(eps, "fp64")
    A.invert()
    b = inputs.rhs_gaussian(Hm.tree.N, 3, 19)
    xi = A.solve(torch.from_numpy(b).to(dev), use_inverse=True).cpu().numpy()
    x_oi = from_tree(Hm, factor.solve(Fz, to_tree(Hm, b), inverse=inv))
    Zd = h2_dense(12, 64, eps)
    xe = from_tree(Hm, np.linalg.solve(Zd, to_tree(Hm, b)))
    print("inverse apply: vs oracle eq. 35 inverse %.2e, vs dense solve %.2e" % (rel(xi, x_oi), rel(xi, xe)))
    assert rel(xi, x_oi) <= 10 * eps
    assert rel(xi, xe) <= 10 * eps
    # mixed-precision factors: the inverse apply refines to the dense solution
    A.factorize(eps, "mixed")
    A.invert()
    xr = A.solve(torch.from_numpy(b).to(dev), use_inverse=True, refine=True, tol=1e-12, max_iter=30).cpu().numpy()
    assert rel(xr, xe) < 1e-10
    A.close()


def test_enomem_and_enoconv(dev):
    from paper_1703_06155_gb300 import H2, H2Error
    eps = 1e-6
    Hm = h2_problem(12, 64, eps)
    rep = oracle_to_rep(Hm)
    with pytest.raises(H2Error) as ei:
        H2.load(rep, arena_cap_bytes=1 << 16)  # the H^2 upload alone needs more
    assert ei.value.status == -2
    A0 = H2.load(rep)
    base = A0.stats()["dev_bytes"]
    A0.close()
    # room for the matrix and a matvec's work buffers (task staging, two
    # vectors), not for the factors (the near-field arena alone is ~9 MB)
    A = H2.load(rep, arena_cap_bytes=base + (4 << 20))
    with pytest.raises(H2Error) as ei:
        A.factorize(eps, "fp64")
    assert ei.value.status == -2 and b"cap" in ei.value.args[0].encode()
    with pytest.raises(H2Error) as ei:
        A.solve(torch.zeros(Hm.tree.N, dtype=torch.complex128, device=dev))
    assert ei.value.status == -8  # no factorization: call out of order
    # the context still multiplies (its H^2 matrix is intact)
    x = inputs.rhs_gaussian(Hm.tree.N, 1, 3)[:, 0]
    y = A.matvec(torch.from_numpy(x).to(dev)).cpu().numpy()
    assert rel(y, from_tree(Hm, oh2.matvec(Hm, to_tree(Hm, x)))) < 1e-13
    A.close()
    # refinement that cannot reach its tolerance: H2_ENOCONV, x = last iterate
    B = H2.load(rep)
    B.factorize(eps, "mixed")
    b = torch.from_numpy(inputs.rhs_gaussian(Hm.tree.N, 1, 7)[:, 0]).to(dev)
    with pytest.raises(H2Error) as ei:
        B.solve(b, refine=True, tol=1e-15, max_iter=0)
    assert ei.value.status == -4
    x = B.solve(b, refine=True, tol=1e-15, max_iter=0, allow_noconv=True)
    assert B.last_solve["status"] == -4 and B.last_solve["iters"] == 0
    assert 1e-15 < B.last_solve["resid"] < 1e-3
    assert rel(x.cpu().numpy(), B.solve(b).cpu().numpy()) < 1e-12  # no correction was applied
    B.close()


def _dense_A(Hm, Zd_tree, chi):
    """A = D^{-1/2} Z D^{1/2} in global order from the tree-order dense Z_H2."""
    p = Hm.tree.perm
    Z = np.empty_like(Zd_tree)
    Z[np.ix_(p, p)] = Zd_tree
    s = np.sqrt(chi)
    return Z * (s[None, :] / s[:, None])


def test_set_chi_matches_dense_rescaled_matrix(dev):
    from paper_1703_06155_gb300 import H2
    eps = 1e-6
    Hm = h2_problem(12, 64, eps, percell_seed=4)
    N = Hm.tree.N
    chi = inputs.chi_random_cells(N, 4)
    Zd = h2_dense(12, 64, eps, percell_seed=4)
    A = H2.load(oracle_to_rep(Hm, dscale=np.sqrt(chi)))
    chi2 = chi * (1.0 + 0.2 * np.random.default_rng(8).random(N))
    A.set_chi(chi2)
    # Z' = I + E (Z - I) E, E = diag(sqrt(chi2 / chi)) in tree order
    e = np.sqrt(chi2 / chi)[Hm.tree.perm]
    Z2 = np.eye(N) + e[:, None] * (Zd - np.eye(N)) * e[None, :]
    A2 = _dense_A(Hm, Z2, chi2)
    x = inputs.rhs_gaussian(N, 2, 21)
    y = A.matvec(torch.from_numpy(x).to(dev)).cpu().numpy()
    assert rel(y, A2 @ x) < 1e-12
    # and Z' is the dense kernel matrix at chi2 to the construction accuracy
    idx = Hm.tree.perm
    Zex = kernel.entries(Hm.pts, chi2, idx, idx, K, H)
    assert rel(Z2, Zex) < 10 * eps
    with pytest.raises(Exception) as ei:
        A.solve(torch.from_numpy(x).to(dev))
    assert getattr(ei.value, "status", None) == -8  # factors were invalidated
    A.factorize(eps, "mixed")
    xs = A.solve(torch.from_numpy(x).to(dev), refine=True, tol=1e-13, max_iter=30).cpu().numpy()
    assert rel(xs, np.linalg.solve(A2, x)) < 1e-10
    A.close()


def test_autograd_step_in_chi_on_one_context(dev):
    # one gradient step in chi: the node moves its context to the new chi
    # (h2_set_chi + refactorization) and the solution equals a dense solve of
    # the rescaled matrix; the gradient at the new chi matches the dense FP64
    # adjoint gradient there
    from paper_1703_06155_gb300 import H2, autograd
    eps = 1e-6
    Hm = h2_problem(12, 64, eps, percell_seed=4)
    N = Hm.tree.N
    pts = Hm.pts
    chi = inputs.chi_random_cells(N, 4)
    Zd = h2_dense(12, 64, eps, percell_seed=4)
    A = H2.load(oracle_to_rep(Hm, dscale=np.sqrt(chi)))
    A.factorize(eps, "mixed")
    b = inputs.rhs_plane_wave(pts, K)
    probes = inputs.fibonacci_sphere(64, pts.mean(axis=0), 2.0 * (np.sqrt(3.0) / 2.0) * 12 * H)
    G = torch.from_numpy(adjoint.probe_matrix(probes, pts, K, H)).to(dev)
    bt = torch.from_numpy(b).to(dev)

    def loss_grad(c_np):
        c = torch.tensor(c_np, dtype=torch.float64, device=dev, requires_grad=True)
        x = autograd.solve(A, c, bt, refine=True, tol=1e-13)
        L = torch.sum(torch.abs(G @ (c * x)) ** 2)
        L.backward()
        return float(L.detach()), c.grad.cpu().numpy(), x.detach().cpu().numpy()

    L0, g0, _ = loss_grad(chi)
    step = 0.05 * np.max(chi) / np.max(np.abs(g0))
    chi1 = chi - step * g0
    assert np.all(chi1 > 0)
    L1, g1, x1 = loss_grad(chi1)
    assert np.array_equal(A.chi, chi1)
    e = np.sqrt(chi1 / chi)[Hm.tree.perm]
    Z1 = np.eye(N) + e[:, None] * (Zd - np.eye(N)) * e[None, :]
    A1 = _dense_A(Hm, Z1, chi1)
    xd = np.linalg.solve(A1, b)
    print("chi step: L %.6e -> %.6e, ||x - x_dense|| / ||x_dense|| = %.2e" % (L0, L1, rel(x1, xd)))
    assert rel(x1, xd) < 1e-10
    assert L1 < L0  # a descent step
    # gradient at chi1 against the oracle's dense FP64 adjoint gradient there
    _, _, gd, _ = adjoint.probe_gradient(A1, None, G.cpu().numpy(), chi1, b, 1.0)
    assert np.max(np.abs(g1 - gd)) <= 1e-8 * np.max(np.abs(gd)), np.max(np.abs(g1 - gd)) / np.max(np.abs(gd))
    A.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_early_stop_matches_oracle(dev, prec):
    # Sec. III-C: stop at a level above l0 and factorize the rest as one dense
    # block.  eps_fill = 0: exact block LU; eps_fill = eps: within 10 eps of the
    # oracle's factorization with the same stop level (FP64), or refined to the
    # dense solution (mixed); the explicit inverse applies the same factors.
    from paper_1703_06155_gb300 import H2
    eps = 1e-6
    Hm = h2_problem(12, 64, eps)
    Zd = h2_dense(12, 64, eps)
    b = inputs.rhs_gaussian(Hm.tree.N, 2, 29)
    bt = torch.from_numpy(b).to(dev)
    xe = from_tree(Hm, np.linalg.solve(Zd, to_tree(Hm, b)))
    A = H2.load(oracle_to_rep(Hm))
    for ls in range(Hm.l0 + 1, Hm.L + 1):
        A.set_opts(stop_level=ls)
        A.factorize(0.0, "fp64")
        assert A.stats()["stop_level"] == ls
        assert rel(A.solve(bt).cpu().numpy(), xe) < 1e-10, ls
        A.factorize(eps, prec)
        if prec == "fp64":
            Fz = factor.factorize(Hm, eps, "colored", stop_level=ls)
            x_orc = from_tree(Hm, factor.solve(Fz, to_tree(Hm, b)))
            x = A.solve(bt).cpu().numpy()
            print("stop level %d: vs oracle %.2e, vs dense %.2e" % (ls, rel(x, x_orc), rel(x, xe)))
            assert rel(x, x_orc) <= 10 * eps
            k0, kt = A.level_ranks(ls)
            assert np.all(np.abs(kt.astype(int) - Fz.levels[-1].kt.astype(int)) <= 1)
        else:
            x = A.solve(bt, refine=True, tol=1e-12, max_iter=30).cpu().numpy()
            assert rel(x, xe) < 1e-10
        A.invert()
        xi = A.solve(bt, use_inverse=True).cpu().numpy()
        assert rel(xi, A.solve(bt).cpu().numpy()) < 1e-12 if prec == "fp64" else 1e-5
    A.close()


def test_rod_workload_parity(dev):
    # the rod of Sec. VI-B (0.4 x 0.4 x 10 wavelengths, h = 0.1, eps_r = 2.54):
    # the oracle's H^2 matrix factorized on the GPU within 10 eps of the
    # oracle's own factorization, and the library's construction of the same
    # rod solved to its exact-matrix residual
    from paper_1703_06155_gb300 import H2
    eps = 1e-4
    pts = inputs.rod_points(10.0, 0.1)
    N = len(pts)
    chi = inputs.chi_uniform(N, 1.54)
    Hm = oh2.build(pts, chi, K, 0.1, leafsize=64, eps=eps)
    Fz = factor.factorize(Hm, eps, "colored")
    b = inputs.rhs_gaussian(N, 1, 3)[:, 0]
    x_orc = from_tree(Hm, factor.solve(Fz, to_tree(Hm, b)))
    A = H2.load(oracle_to_rep(Hm))
    A.factorize(eps, "fp64")
    x = A.solve(torch.from_numpy(b).to(dev)).cpu().numpy()
    print("rod: vs oracle %.2e" % rel(x, x_orc))
    assert rel(x, x_orc) <= 10 * eps
    B = H2.build(pts, K, 0.1, chi, eps)
    B.factorize(eps, "mixed")
    xb = B.solve(torch.from_numpy(b).to(dev), refine=True, tol=1e-10, max_iter=30).cpu().numpy()
    idx = np.arange(N)
    Z = kernel.entries(pts, chi, idx, idx, K, 0.1)
    assert np.linalg.norm(Z @ xb - b) / np.linalg.norm(b) < 10 * eps
    A.close()
    B.close()


def test_proxy_construction_on_gpu(dev):
    # the proxy construction with the far-field Grams on the GPU: the same
    # matrix as the host build to rounding, within 10 eps of the dense kernel
    # matrix, and its factorization refines to the dense solution
    from paper_1703_06155_gb300 import H2
    eps = 1e-6
    pts = inputs.grid_points(16, H)
    N = len(pts)
    chi = inputs.chi_uniform(N, 3.0)
    A = H2.build(pts, K, H, chi, eps, proxy_min=64)
    B = H2.build(pts, K, H, chi, eps, proxy_min=64, host_only=1)
    Za, _ = dense_from_rep(A.export())
    Zb, _ = dense_from_rep(B.export())
    idx = A.export()["perm"]
    Zex = kernel.entries(pts, chi, idx, idx, K, H)
    assert rel(Za, Zex) < 10 * eps and rel(Za, Zb) < 10 * eps
    A.factorize(eps, "mixed")
    b = inputs.rhs_gaussian(N, 2, 41)
    x = A.solve(torch.from_numpy(b).to(dev), refine=True, tol=1e-12, max_iter=30).cpu().numpy()
    Zg = np.empty_like(Zex)
    Zg[np.ix_(idx, idx)] = Zex
    assert np.linalg.norm(Zg @ x - b) / np.linalg.norm(b) < 10 * eps
    A.close()
    B.close()


def test_matvec_emulation_against_fp64_and_oracle(dev):
    # the FP64 H^2 matvec with its products in double-float on the FP32 pipe
    # (h2_opts.matvec_emulation) against FP64 FMAs and the oracle's matvec,
    # and a refined solve whose residuals ran emulated, checked with FP64
    from paper_1703_06155_gb300 import H2
    eps = 1e-6
    Hm = h2_problem(16, 64, eps)
    A = H2.load(oracle_to_rep(Hm))
    N = Hm.tree.N
    x = inputs.rhs_gaussian(N, 4, 3)
    xt = torch.from_numpy(x).to(dev)
    A.set_opts(matvec_emulation=0)
    y64 = A.matvec(xt).cpu().numpy()
    A.set_opts(matvec_emulation=2, profile=1)
    y2 = A.matvec(xt).cpu().numpy()
    paths = A.stats()["paths"]
    y_orc = np.stack([from_tree(Hm, oh2.matvec(Hm, to_tree(Hm, x[:, q]))) for q in range(4)], axis=1)
    e_fp64, e_orc = rel(y2, y64), rel(y2, y_orc)
    print("matvec emulation: vs FP64 FMAs %.2e, vs oracle %.2e (FP64 FMAs vs oracle %.2e)"
          % (e_fp64, e_orc, rel(y64, y_orc)))
    assert any(k.startswith("gemm:fp64_dd:") for k in paths), paths
    assert e_fp64 <= 1e-12 and e_orc <= 1e-12
    # refined solve to 1e-10 with emulated residuals (default 1), residual
    # re-evaluated with FP64 FMAs
    A.set_opts(matvec_emulation=1, profile=0)
    A.factorize(eps, "mixed")
    b = inputs.rhs_gaussian(N, 4, 4)
    bt = torch.from_numpy(b).to(dev)
    xs = A.solve(bt, refine=True, tol=1e-10, max_iter=30)
    res_emul = A.last_solve["resid"]
    A.set_opts(matvec_emulation=0)
    r = A.matvec(xs).cpu().numpy() - b
    res64 = float(np.max(np.linalg.norm(r, axis=0) / np.linalg.norm(b, axis=0)))
    print("refined solve: emulated residual %.2e, FP64 residual %.2e" % (res_emul, res64))
    assert res_emul <= 1e-10 and res64 <= 2e-10
    A.close()


_CHECKED_RUN = r"""
import sys, numpy as np, torch
sys.path[:0] = ["tests", "."]
from _problems import h2_problem
from _h2io import oracle_to_rep
from paper_1703_06155_gb300 import H2, inputs, factorize_batch, solve_batch
H = h2_problem(16, 64, 1e-6)
b = torch.from_numpy(inputs.rhs_gaussian(H.tree.N, 3, 7)).cuda()
A = H2.load(oracle_to_rep(H))
A.factorize(1e-6, "mixed")
A.solve(b, refine=True, tol=1e-10, max_iter=30)
A.factorize(1e-6, "fp64")
A.invert()
A.solve(b, use_inverse=True)
A.solve(b, adjoint=True)
A.matvec(b)
A.set_opts(stop_level=H.l0 + 1)
A.factorize(1e-6, "mixed")
A.solve(b)
cs = [H2.load(oracle_to_rep(h2_problem(n, 64, 1e-6))) for n in (12, 16)]
factorize_batch(cs, 1e-6, "mixed")
solve_batch(cs, [torch.from_numpy(inputs.rhs_gaussian(c.stats()["N"], 2, 3)).cuda() for c in cs], refine=True)
print("checked run ok")
"""


def test_bounds_checked_run(dev):
    # the same library with H2_CHECKS set: every GEMM, copy, apply and
    # partial-LU task list of a mixed and an FP64 factorization (full and
    # early-stopped), refined / adjoint / inverse-based solves, a matvec and
    # a two-instance batch is checked on the host against the allocations it
    # touches before its launch; any overrun would fail the call
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, H2_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", _CHECKED_RUN], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    print(r.stdout[-2000:], r.stderr[-2000:])
    assert r.returncode == 0 and "checked run ok" in r.stdout
