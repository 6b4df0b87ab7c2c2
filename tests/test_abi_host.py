"""CPU-only checks of libh2: it builds, loads, exports every symbol of
include/h2.h, and its host-side planning (cluster tree, partition, H^2
construction with host_only=1) agrees with the oracle / the dense matrix.
No compute call here touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import kernel
from oracle import tree as otree
from paper_1703_06155_gb300 import inputs

from _problems import H, K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libh2():
    from paper_1703_06155_gb300 import _build, lib
    _build.build()
    return lib()


def test_exports_every_declared_symbol(libh2):
    hdr = open(os.path.join(ROOT, "include", "h2.h")).read()
    decl = set(re.findall(r"^(?:h2_status|void|const char\*)\s+(h2_[a-z_]+)\s*\(", hdr, re.M))
    assert len(decl) >= 12
    for name in decl:
        assert hasattr(libh2, name), name
    from paper_1703_06155_gb300 import SYMBOLS
    assert set(SYMBOLS) == decl


def dense_from_rep(r):
    """Assemble Z_H2 (tree order) from the h2_load layout, independently of
    both the oracle and the library."""
    L, l0 = r["L"], r["l0"]
    ranks, o = {}, 0
    for l in range(l0, L + 1):
        ranks[l] = r["rank"][o:o + 2 ** l]
        o += 2 ** l
    sizes = {L: r["leaf_size"]}
    for l in range(L - 1, -1, -1):
        sizes[l] = sizes[l + 1][0::2] + sizes[l + 1][1::2]
    starts = {l: np.concatenate([[0], np.cumsum(sizes[l])[:-1]]) for l in sizes}
    full, o = {}, 0
    for c in range(2 ** L):
        cnt = sizes[L][c] * ranks[L][c]
        full[(L, c)] = r["V"][o:o + cnt].reshape(ranks[L][c], sizes[L][c]).T
        o += cnt
    o = 0
    for l in range(L - 1, l0 - 1, -1):
        pass
    Tm, o = {}, 0
    for l in range(l0, L):
        for c in range(2 ** l):
            k1, k2 = ranks[l + 1][2 * c], ranks[l + 1][2 * c + 1]
            cnt = (k1 + k2) * ranks[l][c]
            Tm[(l, c)] = r["T"][o:o + cnt].reshape(ranks[l][c], k1 + k2).T
            o += cnt
    for l in range(L - 1, l0 - 1, -1):
        for c in range(2 ** l):
            A1, A2 = full[(l + 1, 2 * c)], full[(l + 1, 2 * c + 1)]
            W = np.zeros((A1.shape[0] + A2.shape[0], A1.shape[1] + A2.shape[1]), complex)
            W[:A1.shape[0], :A1.shape[1]] = A1
            W[A1.shape[0]:, A1.shape[1]:] = A2
            full[(l, c)] = W @ Tm[(l, c)]
    N = r["N"]
    Z = np.zeros((N, N), complex)
    adm = r["adm"].reshape(-1, 2)
    o = so = 0
    for i, l in enumerate(range(l0, L + 1)):
        for q in range(r["n_adm"][i]):
            t, s = adm[o]
            o += 1
            cnt = ranks[l][t] * ranks[l][s]
            S = r["S"][so:so + cnt].reshape(ranks[l][s], ranks[l][t]).T
            so += cnt
            Z[starts[l][t]:starts[l][t] + sizes[l][t], starts[l][s]:starts[l][s] + sizes[l][s]] = \
                full[(l, t)] @ S @ full[(l, s)].T
    do = 0
    for t, s in r["near"].reshape(-1, 2):
        cnt = sizes[L][t] * sizes[L][s]
        Z[starts[L][t]:starts[L][t] + sizes[L][t], starts[L][s]:starts[L][s] + sizes[L][s]] = \
            r["D"][do:do + cnt].reshape(sizes[L][s], sizes[L][t]).T
        do += cnt
    return Z, full


@pytest.mark.parametrize("n,eps", [(12, 1e-6), (12, 1e-3)])
def test_host_build_matches_oracle_tree_and_dense(libh2, n, eps):
    from paper_1703_06155_gb300 import H2
    pts = inputs.grid_points(n, H)
    N = len(pts)
    chi = inputs.chi_random_cells(N, 4)
    A = H2.build(pts, K, H, chi, eps, host_only=1)
    r = A.export()
    T = otree.ClusterTree(pts, 64)
    P = otree.Partition(T, 1.0)
    assert np.array_equal(T.perm, r["perm"])
    assert r["L"] == T.L and r["l0"] == P.l0
    adm = [tuple(x) for x in r["adm"].reshape(-1, 2)]
    assert adm == [p for l in range(P.l0, T.L + 1) for p in P.adm[l]]
    near = [tuple(x) for x in r["near"].reshape(-1, 2)]
    assert near == P.inad[T.L]
    assert np.allclose(r["dscale"], np.sqrt(chi))
    Z, full = dense_from_rep(r)
    idx = r["perm"]
    Zex = kernel.entries(pts, chi, idx, idx, K, H)
    assert np.linalg.norm(Z - Zex) / np.linalg.norm(Zex) < 10 * eps
    for (l, c), V in full.items():
        if V.shape[1]:
            assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-12
    # host-only contexts refuse GPU work with H2_ESTATE
    with pytest.raises(Exception) as ei:
        A.factorize(eps)
    assert getattr(ei.value, "status", None) == -8


def test_bad_arguments_are_rejected(libh2):
    from paper_1703_06155_gb300 import H2, H2Error
    pts = inputs.grid_points(4, H)
    with pytest.raises(H2Error) as ei:
        H2.build(pts, K, H, 0.0, 1e-6, host_only=1)  # chi must be > 0
    assert ei.value.status == -1
    with pytest.raises(H2Error):
        H2.build(pts, K, H, 3.0, -1.0, host_only=1)
    out = ctypes.c_void_p()
    assert libh2.h2_factorize(None, 1e-6, 0) == -1
    assert libh2.h2_load(0, 0, 0, None, None, None, None, None, None, None, None, 0, None, None, None, None, None,
                         ctypes.byref(out)) == -1


def test_batch_calls_reject_bad_groups(libh2):
    # no GPU needed: the group checks run before any device work
    from paper_1703_06155_gb300 import H2
    pts = inputs.grid_points(4, H)
    a = H2.build(pts, K, H, 3.0, 1e-6, host_only=1)
    arr = (ctypes.c_void_p * 2)(a._h.value, a._h.value)
    assert libh2.h2_factorize_batch(None, 1, 1e-6, 0) == -1
    assert libh2.h2_factorize_batch(arr, 0, 1e-6, 0) == -1
    assert libh2.h2_factorize_batch(arr, 2, 1e-6, 0) == -1      # the same context twice
    assert libh2.h2_factorize_batch(arr, 1, 1e-6, 0) == -1      # host_only context
    one = (ctypes.c_void_p * 1)(None)
    assert libh2.h2_solve_batch(arr, 1, one, one, 1, 0, 1e-6, 1, None, None, None) == -1
    a.close()


def test_set_opts_validates(libh2):
    from paper_1703_06155_gb300 import H2, H2Error, default_opts
    pts = inputs.grid_points(4, H)
    a = H2.build(pts, K, H, 3.0, 1e-6, host_only=1)
    a.set_opts(apply_path=1, split_target=300, cluster_max=8, tile_policy=1)
    for bad in (dict(apply_path=3), dict(cluster_max=17), dict(tile_policy=2), dict(split_target=-1),
                dict(tensor_cores=3), dict(tensor_cores=-1), dict(gram_emulation=2)):
        with pytest.raises(H2Error):
            a.set_opts(**bad)
    assert libh2.h2_set_opts(None, ctypes.byref(default_opts())) == -1
    # the ctypes mirror of h2_opts reads the library's defaults field by field
    o = default_opts()
    assert (o.leafsize, o.tensor_cores, o.gram_emulation, o.profile) == (64, 2, 1, 0)
    a.close()


@pytest.mark.parametrize("N", [1, 2, 7, 64, 65, 129])
def test_degenerate_sizes_build(libh2, N):
    # one point, fewer points than a leaf, exactly one leaf, one point past a
    # leaf (a ragged split): the host build still matches the oracle's tree and
    # reproduces the dense matrix
    from paper_1703_06155_gb300 import H2
    pts = np.ascontiguousarray(inputs.grid_points(6, H)[:N])
    chi = inputs.chi_uniform(N, 3.0)
    eps = 1e-6
    A = H2.build(pts, K, H, chi, eps, host_only=1)
    r = A.export()
    T = otree.ClusterTree(pts, 64)
    assert np.array_equal(T.perm, r["perm"]) and r["L"] == T.L
    Z, _ = dense_from_rep(r)
    idx = r["perm"]
    Zex = kernel.entries(pts, chi, idx, idx, K, H)
    assert np.linalg.norm(Z - Zex) <= 10 * eps * np.linalg.norm(Zex)
    A.close()
