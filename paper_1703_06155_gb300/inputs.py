"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only draws and lays out inputs: regular-grid collocation points,
per-cell contrast values and right-hand sides.  It holds none of the solver's
arithmetic (no kernel entries, no factorization, no H^2 construction), so that
the oracle and the product path can both take their inputs from it without
sharing any of the method.

Workload recipe (a scalar stand-in for the paper's SWG volume-integral-equation
matrices of Section VI): points are cell centres of an n x n x n grid of spacing
h filling a cube; global index i + n*(j + n*l); wavenumber k = 2*pi (lambda=1).
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def grid_points(n, h=1.0 / 16.0):
    """Cell centres ((i+1/2)h, (j+1/2)h, (l+1/2)h), index i + n*(j + n*l).

    Returns an (n**3, 3) float64 array, row-major (x, y, z per row).
    """
    c = (np.arange(n, dtype=np.float64) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).copy()


def rod_points(length, h=0.1, side=0.4):
    """Cell centres of a dielectric rod: a (side x side x length) box of cells of
    edge h (wavelength units), index i + nx*(j + nx*l), nx = round(side / h).
    The rod workload of Sec. VI-B (cross-section 0.4 x 0.4 wavelengths, mesh
    0.1 wavelength, length growing) on a regular grid."""
    nx = int(round(side / h))
    nz = int(round(length / h))
    cx = (np.arange(nx, dtype=np.float64) + 0.5) * h
    cz = (np.arange(nz, dtype=np.float64) + 0.5) * h
    z, y, x = np.meshgrid(cz, cx, cx, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).copy()


def chi_uniform(N, chi):
    """Uniform contrast chi = eps_r - 1 for all N cells."""
    return np.full(N, float(chi), dtype=np.float64)


def chi_random_cells(N, seed, lo=1.5, hi=2.0):
    """Per-cell contrast chi_i = lo + (hi-lo)*U(0,1) drawn with PCG64(seed)."""
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random(N)


def rhs_gaussian(N, nrhs, seed):
    """Column-major N x nrhs complex128 RHS, re and im i.i.d. N(0,1) (PCG64)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((nrhs, N))
    im = rng.standard_normal((nrhs, N))
    # stored as (nrhs, N) row-major == (N, nrhs) column-major
    return np.ascontiguousarray((re + 1j * im).T.copy(order="F"))


def rhs_plane_wave(points, k=TWO_PI):
    """Incident plane wave b_i = exp(-j k z_i) (one column)."""
    return np.exp(-1j * k * points[:, 2]).astype(np.complex128)


def fibonacci_sphere(count, centre, radius):
    """`count` golden-angle (Fibonacci) points on a sphere (used for probes)."""
    i = np.arange(count, dtype=np.float64) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / count)
    theta = math.pi * (1.0 + 5.0 ** 0.5) * i
    pts = np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], axis=1)
    return np.asarray(centre, dtype=np.float64)[None, :] + radius * pts


# Named workloads (grid edge, spacing, contrast, epsilon, nrhs, seed).
WORKLOADS = {
    "grid16_fp64": dict(n=16, h=1.0 / 16, chi=3.0, eps=1e-6, nrhs=1, seed=0),
    "grid32": dict(n=32, h=1.0 / 16, chi=3.0, eps=1e-6, nrhs=16, seed=1),
    "grid32_eps1e-4": dict(n=32, h=1.0 / 16, chi=3.0, eps=1e-4, nrhs=16, seed=1),
    "grid96": dict(n=96, h=1.0 / 16, chi=1.5, eps=1e-4, nrhs=4, seed=2),
    "grid48_adjoint": dict(n=48, h=1.0 / 16, chi=None, eps=1e-6, nrhs=1, seed=4),
}
