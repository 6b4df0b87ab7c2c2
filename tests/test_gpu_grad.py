"""Derivative of the GPU solve in the per-cell contrast (autograd node over
h2_solve / h2_solve(H2_ADJOINT) / h2_grad_chi) against

  * the FP64 dense adjoint gradient of the oracle (exact kernel, dense LU);
  * central finite differences (step 1e-6) of the same H^2 system on 8 random
    cells, each perturbed solve refined with the unperturbed factors against
    A' x = A x + (delta / chi_i) (A e_i - e_i) x_i down to a 1e-13 residual,
    so that the difference quotient carries ~1e-7 relative noise.

Workload: 12^3 cells, k = 2 pi, h = 1/16, chi_i = 1.5 + 0.5 U(0, 1), incident
plane wave b = exp(-j k z), L = sum over 64 Fibonacci-sphere probes (radius
twice the cube's half-diagonal) of |E|^2, E = G_E D_chi x.  Gate: 1e-4
relative (to the largest |dL/dchi|).
"""
import math

import numpy as np
import pytest

from oracle import adjoint, kernel
from paper_1703_06155_gb300 import inputs

from _h2io import oracle_to_rep
from _problems import H, K, h2_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SIDE, SEED, EPS = 12, 4, 1e-6


@pytest.fixture(scope="module")
def setup():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1703_06155_gb300 import H2
    dev = torch.device("cuda:0")
    pts = inputs.grid_points(N_SIDE, H)
    N = len(pts)
    chi = inputs.chi_random_cells(N, SEED)
    b = inputs.rhs_plane_wave(pts, K)
    radius = 2.0 * (math.sqrt(3.0) / 2.0) * N_SIDE * H
    probes = inputs.fibonacci_sphere(64, pts.mean(axis=0), radius)
    G = adjoint.probe_matrix(probes, pts, K, H)
    Hh = h2_problem(N_SIDE, 64, EPS, percell_seed=SEED)
    ctx = H2.load(oracle_to_rep(Hh, dscale=np.sqrt(chi)))
    ctx.factorize(EPS, "mixed")
    return dict(dev=dev, pts=pts, chi=chi, b=b, G=G, ctx=ctx)


def gpu_gradient(s):
    from paper_1703_06155_gb300 import autograd
    dev = s["dev"]
    chi_t = torch.tensor(s["chi"], dtype=torch.float64, device=dev, requires_grad=True)
    b_t = torch.from_numpy(s["b"]).to(dev)
    G_t = torch.from_numpy(s["G"]).to(dev)
    x = autograd.solve(s["ctx"], chi_t, b_t, refine=True, tol=1e-12)
    E = G_t @ (chi_t * x)
    L = torch.sum(torch.abs(E) ** 2)
    L.backward()
    return float(L.detach()), chi_t.grad.cpu().numpy(), x.detach().cpu().numpy()


def test_gradient_matches_dense_adjoint(setup):
    s = setup
    _, g, x = gpu_gradient(s)
    A = kernel.dense_A(s["pts"], s["chi"], K, H)
    x_ref, _, red, _ = adjoint.probe_gradient(A, None, s["G"], s["chi"], s["b"], 1.0)
    err_x = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    err = np.max(np.abs(g - red)) / np.max(np.abs(red))
    print("x vs dense: %.3e   grad vs dense adjoint: %.3e" % (err_x, err))
    assert err_x < 1e-4
    assert err < 1e-4


def test_gradient_matches_finite_differences(setup):
    s = setup
    ctx, dev = s["ctx"], s["dev"]
    _, g, _ = gpu_gradient(s)
    N = len(s["chi"])
    chi = s["chi"]
    b_t = torch.from_numpy(s["b"]).to(dev)
    G_t = torch.from_numpy(s["G"]).to(dev)
    chi_t = torch.from_numpy(chi).to(dev)
    cells = np.random.default_rng(SEED).choice(N, 8, replace=False)
    nb = float(torch.linalg.norm(b_t))

    def objective(i, d):
        e = torch.zeros(N, dtype=torch.complex128, device=dev)
        e[i] = 1.0
        col = ctx.matvec(e) - e  # (A - I) e_i
        x = ctx.solve(b_t, refine=True, tol=1e-12)
        for _ in range(40):
            r = b_t - ctx.matvec(x) - (d / chi[i]) * col * x[i]
            if float(torch.linalg.norm(r)) <= 1e-13 * nb:
                break
            x = x + ctx.solve(r)
        else:
            raise AssertionError("perturbed refinement did not reach 1e-13")
        c = chi_t.clone()
        c[i] += d
        return float(torch.sum(torch.abs(G_t @ (c * x)) ** 2))

    delta = 1e-6
    fd = np.array([(objective(i, delta) - objective(i, -delta)) / (2 * delta) for i in cells])
    err = np.max(np.abs(fd - g[cells])) / np.max(np.abs(g))
    print("grad vs central differences on 8 cells: %.3e" % err)
    assert err < 1e-4


def test_grad_chi_kernel_forms(setup):
    # h2_grad_chi against its definition on random vectors, several columns,
    # with and without g, accumulate flag
    s = setup
    ctx, dev = s["ctx"], s["dev"]
    N = len(s["chi"])
    rng = np.random.default_rng(7)
    x, mu, g = (rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3)) for _ in range(3))
    ref = adjoint.grad_reduced(s["chi"], x, mu, g)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    got = ctx.grad_chi(T(x), T(mu), T(g)).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    ref0 = 2.0 * adjoint.grad_reduced(s["chi"], x, mu)
    out = torch.zeros(N, dtype=torch.float64, device=dev)
    ctx.grad_chi(T(x), T(mu), None, alpha=2.0, out=out)
    ctx.grad_chi(T(x), T(mu), None, alpha=2.0, out=out, accumulate=True)
    assert np.max(np.abs(out.cpu().numpy() - 2 * ref0)) <= 1e-13 * np.max(np.abs(ref0))
