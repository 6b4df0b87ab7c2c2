"""Derivative of the solve with respect to the per-cell contrast (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper differentiates nothing; the solver's adjoint traversal (the
conjugate-transposed Algorithms 5-6, eqs. 36-42) is what a reverse-mode
derivative of x = A(chi)^{-1} b needs.  Here everything is dense FP64 and
written from the definition:

  A(chi) = I + s K D_chi,  dA/dchi_i = s K e_i e_i^T,
  dx = -A^{-1} (dA) x,     dL = Re sum conj(g) dx   (g: gradient of L in x,
                                                     conjugate-Wirtinger)
  =>  dL/dchi_i = -Re( conj((s K^H mu)_i) x_i ),    A^H mu = g.      (general)

Because A^H = I + D_chi s K^H, (s K^H mu)_i = (g_i - mu_i) / chi_i, so

      dL/dchi_i = Re( x_i conj(mu_i - g_i) ) / chi_i.                 (reduced)

The scattered-field objective of the gradient workload,
E = s G_E D_chi x with G_E[p, i] = k^2 h^3 e^{-jk|p - r_i|} / (4 pi |p - r_i|)
at probe points p and L = sum_p |E_p|^2, depends on chi also outside the
solve.  With w = s G_E^H E and A^H lambda = D_chi w its total derivative is
2 Re( x_i conj(w_i - (s K^H lambda)_i) ), which reduces the same way to
2 Re( x_i conj(lambda_i) ) / chi_i.

All parity is pinned by the tests against central finite differences of
dense solves and against a one-unknown closed form.
"""
import math

import numpy as np

from . import dense as _dense
from . import kernel as _kernel


def dense_K(pts, k, h):
    """K (without the contrast or sign): A(chi = 1, s = 1) - I."""
    N = len(pts)
    idx = np.arange(N)
    return _kernel.entries(pts, np.ones(N), idx, idx, k, h, 1.0) - np.eye(N)


def probe_matrix(probes, pts, k, h):
    """G_E[p, i] = k^2 h^3 e^{-jk r} / (4 pi r), r = |probe_p - point_i|."""
    d = probes[:, None, :] - pts[None, :, :]
    r = np.sqrt(np.sum(d * d, axis=2))
    return (k * k * h ** 3) * np.exp(-1j * k * r) / (4.0 * math.pi * r)


def grad_general(K, sign, x, mu):
    """dL/dchi_i = -Re(conj((s K^H mu)_i) x_i), summed over columns (general form)."""
    x = x.reshape(len(x), -1)
    mu = mu.reshape(len(mu), -1)
    t = sign * (K.conj().T @ mu)
    return -np.sum(np.real(np.conj(t) * x), axis=1)


def grad_reduced(chi, x, mu, g=None):
    """dL/dchi_i = Re(x_i conj(mu_i - g_i)) / chi_i, summed over columns."""
    x = x.reshape(len(x), -1)
    d = mu.reshape(len(mu), -1) - (0 if g is None else g.reshape(len(g), -1))
    return np.sum(np.real(x * np.conj(d)), axis=1) / chi


def probe_objective(G_E, chi, x, sign):
    """L = sum_p |E_p|^2 with E = s G_E D_chi x; returns (L, E)."""
    E = sign * (G_E @ (chi * x))
    return float(np.sum(np.abs(E) ** 2)), E


def probe_gradient(A, K, G_E, chi, b, sign):
    """Total dL/dchi of the probe objective by the adjoint, both forms.

    Returns (x, lambda, grad_reduced, grad_general):
      x = A^{-1} b, w = s G_E^H E, A^H lambda = D_chi w,
      reduced: 2 Re(x conj(lambda)) / chi
      general: 2 Re(x conj(w - s K^H lambda))  (None if K is None).
    One LU of A serves both solves."""
    LU, piv = _dense.lu(A)
    x = _dense.lu_solve(LU, piv, b)
    _, E = probe_objective(G_E, chi, x, sign)
    w = sign * (G_E.conj().T @ E)
    lam = _dense.lu_solve_adjoint(LU, piv, chi * w)
    red = 2.0 * np.real(x * np.conj(lam)) / chi
    gen = None if K is None else 2.0 * np.real(x * np.conj(w - sign * (K.conj().T @ lam)))
    return x, lam, red, gen


def probe_fd(pts, chi, k, h, b, G_E, cells, delta, sign=1.0):
    """Central finite differences of the probe objective in chi at `cells`
    (dense solves of A(chi +- delta e_i) x = b)."""
    out = []
    for i in cells:
        vals = []
        for sgn in (1.0, -1.0):
            c = chi.copy()
            c[i] += sgn * delta
            A = _kernel.dense_A(pts, c, k, h, sign)
            x = _dense.solve(A, b)
            vals.append(probe_objective(G_E, c, x, sign)[0])
        out.append((vals[0] - vals[1]) / (2.0 * delta))
    return np.array(out)
