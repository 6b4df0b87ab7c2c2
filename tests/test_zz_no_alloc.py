"""h2_matvec_noalloc against h2_matvec through the C ABI (GPU).

Some callers cannot allocate device memory at the time they need the H^2
product (their memory is reserved up front, or they run in a loop that must
not call the allocator); h2_matvec_noalloc serves them from a static device
array.  Its result must equal h2_matvec's within the matvec tolerance of the
parity tests (1e-13 relative), call after call, since every call reuses the
same array.  The first calls go to a freshly loaded context, before any
h2_matvec has sized that context's own work buffers, and the context's device
byte count must not move across them.  This file is collected last, so a run
that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from paper_1703_06155_gb300 import inputs

from _h2io import oracle_to_rep
from _problems import h2_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call(fn, h, x, y, nrhs, flags):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), nrhs, flags, stream)


def _rhs(N, nrhs, seed):
    # (nrhs, N) row-major == N x nrhs column-major
    return torch.from_numpy(inputs.rhs_gaussian(N, nrhs, seed).T.copy()).cuda()


def test_noalloc_matvec_matches_matvec_twice():
    from paper_1703_06155_gb300 import H2, lib
    assert torch.cuda.is_available()
    L = lib()
    H = h2_problem(12, 64, 1e-6)
    A = H2.load(oracle_to_rep(H))
    N = H.tree.N
    nrhs = 3
    # fresh context: the allocation-free product first, twice in a row
    dev0 = A.stats()["dev_bytes"]
    ys = {}
    for flags in (0, 1):  # plain product, then the adjoint product (H2_ADJOINT)
        for seed in (3, 4):  # two calls in a row, different inputs
            x = _rhs(N, nrhs, seed)
            y = torch.full_like(x, complex(float("nan"), float("nan")))
            assert _call(L.h2_matvec_noalloc, A._h, x, y, nrhs, flags) == 0, L.h2_last_error(A._h)
            ys[(flags, seed)] = (x, y)
    torch.cuda.synchronize()
    assert A.stats()["dev_bytes"] == dev0
    # then the allocating product on the same inputs
    for (flags, seed), (x, y) in ys.items():
        y_ref = torch.empty_like(x)
        assert _call(L.h2_matvec, A._h, x, y_ref, nrhs, flags) == 0
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref)).item()
        assert err < 1e-13, (flags, seed, err)
    # two more calls after h2_matvec has run: same results, no device bytes
    dev1 = A.stats()["dev_bytes"]
    for flags in (0, 1):
        x, y0 = ys[(flags, 3)]
        y = torch.zeros_like(x)
        assert _call(L.h2_matvec_noalloc, A._h, x, y, nrhs, flags) == 0, L.h2_last_error(A._h)
        torch.cuda.synchronize()
        assert torch.equal(y, y0)
    assert A.stats()["dev_bytes"] == dev1
    # sizes beyond the static array are rejected with a message, not run
    big = 4096
    x = torch.zeros((big, N), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    st = _call(L.h2_matvec_noalloc, A._h, x, y, big, 0)
    assert st == -1
    assert b"static scratch" in L.h2_last_error(A._h)
    # host buffers are rejected (H2_EINVAL), nothing runs
    xh = np.zeros((nrhs, N), np.complex128)
    yh = np.zeros_like(xh)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.h2_matvec_noalloc(A._h, xh.ctypes.data_as(ctypes.c_void_p), yh.ctypes.data_as(ctypes.c_void_p), nrhs, 0,
                             stream)
    assert st == -1
    assert b"device" in L.h2_last_error(A._h)
    A.close()
