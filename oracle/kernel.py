"""Matrix entries of the scalar VIE-like stand-in workload (oracle side).

The paper solves SWG vector VIEs (Sec. VI); this build substitutes a scalar
point-collocation kernel on a regular grid:

  K_ij = k^2 h^3 exp(-j k r_ij) / (4 pi r_ij),                 i != j
  K_ii = k^2 * integral over a ball of radius a (equal volume h^3) of
         exp(-j k r) / (4 pi r) dV = (1 + j k a) exp(-j k a) - 1

and the system matrix A = I + s K D_chi (s = +1, D_chi = diag(chi)).  The
factorized matrix is the diagonally similar, complex-symmetric

  Z = D^{1/2} A D^{-1/2} = I + s D^{1/2} K D^{1/2},

so A x = b  <=>  Z (D^{1/2} x) = D^{1/2} b.
"""
import math

import numpy as np


def ball_radius(h):
    """Radius of the ball with the volume of one cell, a = (3/(4 pi))^(1/3) h."""
    return (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0) * h


def self_term(k, h):
    """Closed form of k^2 * int_{|r|<a} e^{-jkr}/(4 pi r) dV = (1+jka)e^{-jka} - 1."""
    x = k * ball_radius(h)
    return (1.0 + 1j * x) * np.exp(-1j * x) - 1.0


def entries(pts, chi, rows, cols, k, h, sign=1.0):
    """Dense sub-block Z[rows, cols] of Z = I + s D^{1/2} K D^{1/2}.

    rows/cols are integer arrays of global point indices.
    """
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    d = pts[rows][:, None, :] - pts[cols][None, :, :]
    r = np.sqrt(np.sum(d * d, axis=2))
    same = rows[:, None] == cols[None, :]
    r_safe = np.where(same, 1.0, r)
    g = (k * k * h ** 3) * np.exp(-1j * k * r_safe) / (4.0 * math.pi * r_safe)
    sc = np.sqrt(chi[rows])[:, None] * np.sqrt(chi[cols])[None, :]
    z = sign * sc * g
    if np.any(same):
        diag = 1.0 + sign * chi[rows] * self_term(k, h)
        z = np.where(same, diag[:, None] * np.ones((1, len(cols))), z)
    return z.astype(np.complex128)


def dense_A(pts, chi, k, h, sign=1.0):
    """The unscaled system matrix A = I + s K D_chi (global index order)."""
    N = len(pts)
    idx = np.arange(N)
    Z = entries(pts, np.ones(N), idx, idx, k, h, sign)  # I + sK
    K = (Z - np.eye(N)) / sign
    return np.eye(N) + sign * K * chi[None, :]
