"""Small seeded problems shared by the oracle and GPU tests (cached per process)."""
import functools
import math

import numpy as np

from paper_1703_06155_gb300 import inputs

K = 2.0 * math.pi
H = 1.0 / 16.0


@functools.lru_cache(maxsize=None)
def h2_problem(n, leaf, eps, chi=3.0, percell_seed=None):
    from oracle import h2
    pts = inputs.grid_points(n, H)
    N = len(pts)
    c = inputs.chi_uniform(N, chi) if percell_seed is None else inputs.chi_random_cells(N, percell_seed)
    return h2.build(pts, c, K, H, leafsize=leaf, eps=eps)


@functools.lru_cache(maxsize=None)
def h2_dense(n, leaf, eps, chi=3.0, percell_seed=None):
    from oracle import h2
    return h2.dense(h2_problem(n, leaf, eps, chi, percell_seed))


@functools.lru_cache(maxsize=None)
def factorization(n, leaf, eps_build, eps_fill, ordering="colored", chi=3.0, percell_seed=None):
    from oracle import factor
    return factor.factorize(h2_problem(n, leaf, eps_build, chi, percell_seed), eps_fill, ordering)
