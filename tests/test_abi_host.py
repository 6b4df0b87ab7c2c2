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

from _h2io import dense_from_rep
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
                dict(tensor_cores=3), dict(tensor_cores=-1), dict(gram_emulation=2), dict(eig_solver=3),
                dict(matvec_emulation=3), dict(ldlt=3), dict(ldlt=-1)):
        with pytest.raises(H2Error):
            a.set_opts(**bad)
    assert libh2.h2_set_opts(None, ctypes.byref(default_opts())) == -1
    # the ctypes mirror of h2_opts reads the library's defaults field by field
    o = default_opts()
    assert (o.leafsize, o.tensor_cores, o.gram_emulation, o.profile) == (64, 2, 1, 0)
    # the last fields of the struct (a layout mismatch would misread them)
    assert (o.eig_solver, o.matvec_emulation, o.ldlt) == (2, 1, 2)
    a.set_opts(ldlt=0)
    a.set_opts(ldlt=1)
    assert a.stats()["ldlt"] == 0  # no factorization yet
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


def test_set_chi_host_rescale_is_exact(libh2):
    # h2_set_chi on a host_only context (no GPU): the representation becomes
    # I + E (Z - I) E exactly, E = diag(sqrt(chi'/chi)), with the same ranks and
    # orthonormal nested bases; bad contrasts are rejected and change nothing
    from paper_1703_06155_gb300 import H2, H2Error
    pts = inputs.grid_points(8, H)
    N = len(pts)
    chi = inputs.chi_random_cells(N, 4)
    A = H2.build(pts, K, H, chi, 1e-6, leafsize=32, host_only=1)
    r0 = A.export()
    Z0, _ = dense_from_rep(r0)
    chi2 = chi * (1.0 + 0.5 * np.random.default_rng(2).random(N))
    A.set_chi(chi2)
    r1 = A.export()
    Z1, full = dense_from_rep(r1)
    e = np.sqrt(chi2 / chi)[r0["perm"]]
    ref = np.eye(N) + e[:, None] * (Z0 - np.eye(N)) * e[None, :]
    assert np.linalg.norm(Z1 - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.array_equal(r0["rank"], r1["rank"])
    assert np.allclose(r1["dscale"], np.sqrt(chi2), rtol=1e-15, atol=0)
    for V in full.values():
        if V.shape[1]:
            assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-12
    for bad in (np.zeros(N), -chi, np.full(N, np.nan), chi[:5]):
        with pytest.raises(H2Error) as ei:
            A.set_chi(bad)
        assert ei.value.status == -1
    assert np.array_equal(A.export()["S"], r1["S"])
    A.close()


@pytest.mark.parametrize("n,eps", [(12, 1e-6), (16, 1e-4)])
def test_proxy_construction_matches_dense(libh2, n, eps):
    # the proxy-point construction (far field sampled exactly inside three
    # cluster radii, through direction-filtered proxy points beyond) keeps the
    # construction accuracy (<= 10 eps against the dense kernel matrix) and
    # ranks close to those of the exact far-field sample
    from paper_1703_06155_gb300 import H2
    pts = inputs.grid_points(n, H)
    N = len(pts)
    chi = inputs.chi_random_cells(N, 4)
    Ap = H2.build(pts, K, H, chi, eps, host_only=1, proxy_min=64)
    Ae = H2.build(pts, K, H, chi, eps, host_only=1)
    rp, re_ = Ap.export(), Ae.export()
    Zp, full = dense_from_rep(rp)
    idx = rp["perm"]
    Zex = kernel.entries(pts, chi, idx, idx, K, H)
    assert np.linalg.norm(Zp - Zex) <= 10 * eps * np.linalg.norm(Zex)
    for V in full.values():
        if V.shape[1]:
            assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-12
    kp, ke = Ap.stats()["build_rank_max"], Ae.stats()["build_rank_max"]
    assert all(a <= 1.15 * b + 4 for a, b in zip(kp, ke)), (kp, ke)
    Ap.close()
    Ae.close()
