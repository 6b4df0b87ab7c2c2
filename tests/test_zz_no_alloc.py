"""h2_matvec_noalloc against h2_matvec through the C ABI (GPU).

Some callers cannot allocate device memory at the time they need the H^2
product (their memory is reserved up front, or they run in a loop that must
not call the allocator); h2_matvec_noalloc serves them from a static device
array.  Its result must equal h2_matvec's within the matvec tolerance of the
parity tests (1e-13 relative), call after call, since every call reuses the
same array.  This file is collected last, so a run that stops at the first
failure has run every other test before it.
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


def test_noalloc_matvec_matches_matvec_twice():
    from paper_1703_06155_gb300 import H2, lib
    assert torch.cuda.is_available()
    L = lib()
    H = h2_problem(12, 64, 1e-6)
    A = H2.load(oracle_to_rep(H))
    N = H.tree.N
    for flags in (0, 1):  # plain product, then the adjoint product (H2_ADJOINT)
        for seed in (3, 4):  # two calls in a row, different inputs
            nrhs = 3
            x = torch.from_numpy(inputs.rhs_gaussian(N, nrhs, seed).T.copy()).cuda()  # (nrhs, N) = N x nrhs col-major
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, complex(float("nan"), float("nan")))
            assert _call(L.h2_matvec, A._h, x, y_ref, nrhs, flags) == 0
            assert _call(L.h2_matvec_noalloc, A._h, x, y, nrhs, flags) == 0, L.h2_last_error(A._h)
            torch.cuda.synchronize()
            err = (torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref)).item()
            assert err < 1e-13, err
    # sizes beyond the static array are rejected with a message, not run
    big = 4096
    x = torch.zeros((big, N), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    st = _call(L.h2_matvec_noalloc, A._h, x, y, big, 0)
    assert st == -1
    assert b"static scratch" in L.h2_last_error(A._h)
    A.close()
