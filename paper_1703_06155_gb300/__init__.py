"""Python binding of libh2: the accuracy-controlled H^2 direct solver on GB300.

Argument marshalling only: every step of the build, factorization, solve and
matvec runs inside libh2.so (C ABI in include/h2.h).  If the shared library
is missing the import of `H2` fails loudly; there is no Python fallback.

Vectors are complex128 of shape (N,) or (N, nrhs) in the caller's point
order: torch CUDA tensors (device path) or numpy arrays (host path, H2_HOST).
"""
import ctypes
import json
import os

import numpy as np

from . import inputs  # noqa: F401  (seeded workload generators)

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libh2.so")

H2_OK, H2_EINVAL, H2_ENOMEM, H2_ESINGULAR, H2_ENOCONV = 0, -1, -2, -3, -4
H2_ETIMEOUT, H2_ECUDA, H2_EINTERNAL, H2_ESTATE = -5, -6, -7, -8
H2_FP64, H2_MIXED = 0, 1
H2_ADJOINT, H2_REFINE, H2_USE_INVERSE, H2_HOST = 1, 2, 4, 8
H2_GRAD_ACCUMULATE = 1
SYMBOLS = ("h2_default_opts", "h2_build", "h2_load", "h2_factorize", "h2_invert", "h2_solve", "h2_matvec",
           "h2_matvec_noalloc", "h2_factorize_batch", "h2_solve_batch", "h2_grad_chi", "h2_set_opts",
           "h2_set_chi", "h2_level_ranks", "h2_export_sizes", "h2_export", "h2_stats", "h2_last_error",
           "h2_status_string", "h2_destroy")


class h2_opts(ctypes.Structure):
    _fields_ = [("leafsize", ctypes.c_int), ("eta", ctypes.c_double), ("sign", ctypes.c_double),
                ("ordering", ctypes.c_int), ("proxy_min", ctypes.c_int), ("proxy_radius", ctypes.c_double),
                ("arena_cap_bytes", ctypes.c_size_t),
                ("host_only", ctypes.c_int), ("profile", ctypes.c_int), ("apply_path", ctypes.c_int),
                ("solve_graph", ctypes.c_int), ("split_target", ctypes.c_int), ("cluster_max", ctypes.c_int),
                ("tile_policy", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("gram_emulation", ctypes.c_int), ("eig_solver", ctypes.c_int), ("stop_level", ctypes.c_int),
                ("proxy_margin", ctypes.c_double), ("matvec_emulation", ctypes.c_int),
                ("ldlt", ctypes.c_int)]


class H2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


_lib = None


def lib():
    """Load libh2.so (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libh2.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'`"
                          % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.h2_default_opts.argtypes = [ctypes.POINTER(h2_opts)]
    L.h2_default_opts.restype = None
    L.h2_build.argtypes = [P, I64, D, D, P, I64, D, ctypes.POINTER(h2_opts), P, ctypes.POINTER(P)]
    L.h2_load.argtypes = [I64, I, I, P, P, P, P, P, P, P, P, I64, P, P, P, ctypes.POINTER(h2_opts), P,
                          ctypes.POINTER(P)]
    L.h2_factorize.argtypes = [P, D, I]
    L.h2_invert.argtypes = [P]
    L.h2_solve.argtypes = [P, P, P, I, ctypes.c_uint, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    L.h2_matvec.argtypes = [P, P, P, I, ctypes.c_uint, P]
    L.h2_matvec_noalloc.argtypes = [P, P, P, I, ctypes.c_uint, P]
    L.h2_grad_chi.argtypes = [P, P, P, P, I, D, P, ctypes.c_uint, P]
    L.h2_factorize_batch.argtypes = [P, I, D, I]
    L.h2_set_opts.argtypes = [P, ctypes.POINTER(h2_opts)]
    L.h2_set_chi.argtypes = [P, P, I64]
    L.h2_level_ranks.argtypes = [P, I, P, P, I64]
    L.h2_solve_batch.argtypes = [P, I, P, P, I, ctypes.c_uint, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    L.h2_export_sizes.argtypes = [P] + [ctypes.POINTER(I64), ctypes.POINTER(I), ctypes.POINTER(I)] + \
        [ctypes.POINTER(I64)] * 6
    L.h2_export.argtypes = [P] * 12
    L.h2_stats.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t]
    L.h2_last_error.argtypes = [P]
    L.h2_last_error.restype = ctypes.c_char_p
    L.h2_status_string.argtypes = [I]
    L.h2_status_string.restype = ctypes.c_char_p
    L.h2_destroy.argtypes = [P]
    L.h2_destroy.restype = None
    for name in ("h2_build", "h2_load", "h2_factorize", "h2_invert", "h2_solve", "h2_matvec", "h2_matvec_noalloc",
                 "h2_grad_chi", "h2_factorize_batch", "h2_solve_batch", "h2_set_opts", "h2_set_chi", "h2_level_ranks",
                 "h2_export_sizes", "h2_export", "h2_stats"):
        getattr(L, name).restype = I
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def default_opts(**kw):
    o = h2_opts()
    lib().h2_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "ordering" and isinstance(v, str):
            v = {"colored": 0, "natural": 1}[v]
        setattr(o, k, v)
    return o


class H2:
    """An H^2 matrix on the GPU with its factorization (one libh2 context)."""

    def __init__(self, handle, chi=None):
        self._h = handle
        self.N = self._sizes()[0]
        # the contrast the context was set up with (host float64, length N)
        self.chi = None if chi is None else np.broadcast_to(np.asarray(chi, np.float64), (self.N,)).copy()

    # ---------------------------------------------------------------- setup
    @classmethod
    def build(cls, points, k, h, chi, eps, stream=None, **opts):
        """h2_build from HOST points (N x 3) and chi (N or scalar)."""
        pts = np.ascontiguousarray(points, dtype=np.float64)
        c = np.ascontiguousarray(np.atleast_1d(np.asarray(chi, dtype=np.float64)))
        o = default_opts(**opts)
        out = ctypes.c_void_p()
        st = lib().h2_build(_ptr(pts), len(pts), float(k), float(h), _ptr(c), len(c), float(eps), ctypes.byref(o),
                            _stream(stream), ctypes.byref(out))
        if st != H2_OK:
            raise H2Error(st, "h2_build: " + lib().h2_last_error(None).decode())
        return cls(out, chi=c)

    @classmethod
    def load(cls, rep, stream=None, **opts):
        """h2_load from a dict of host arrays in the layout of `export()`."""
        r = {k: (np.ascontiguousarray(v) if isinstance(v, np.ndarray) else v) for k, v in rep.items()}
        o = default_opts(**opts)
        out = ctypes.c_void_p()

        def cplx(a):
            return None if a is None or len(a) == 0 else np.ascontiguousarray(a, dtype=np.complex128)

        V, T, S, D = cplx(r["V"]), cplx(r["T"]), cplx(r["S"]), cplx(r["D"])
        keep = [V, T, S, D]
        st = lib().h2_load(int(r["N"]), int(r["L"]), int(r["l0"]), _ptr(r["perm"].astype(np.int64)),
                           _ptr(r["leaf_size"].astype(np.int64)), _ptr(r["rank"].astype(np.int64)), _ptr(V),
                           _ptr(T), _ptr(r["n_adm"].astype(np.int64)), _ptr(r["adm"].astype(np.int64)), _ptr(S),
                           int(len(r["near"]) // 2), _ptr(r["near"].astype(np.int64)), _ptr(D),
                           _ptr(r.get("dscale")), ctypes.byref(o), _stream(stream), ctypes.byref(out))
        del keep
        if st != H2_OK:
            raise H2Error(st, "h2_load: " + lib().h2_last_error(None).decode())
        ds = r.get("dscale")
        # h2_load takes dscale = sqrt(chi); without it the columns are unscaled (chi = 1)
        return cls(out, chi=1.0 if ds is None else np.asarray(ds, np.float64) ** 2)

    def _check(self, st, what):
        if st != H2_OK:
            raise H2Error(st, "%s: %s" % (what, lib().h2_last_error(self._h).decode()))

    def _sizes(self):
        N, nV, nT, nS, na, nn, nD = (ctypes.c_int64() for _ in range(7))
        L, l0 = ctypes.c_int(), ctypes.c_int()
        lib().h2_export_sizes(self._h, ctypes.byref(N), ctypes.byref(L), ctypes.byref(l0), ctypes.byref(nV),
                              ctypes.byref(nT), ctypes.byref(nS), ctypes.byref(na), ctypes.byref(nn),
                              ctypes.byref(nD))
        return N.value, L.value, l0.value, nV.value, nT.value, nS.value, na.value, nn.value, nD.value

    def export(self):
        """The H^2 representation as host arrays (h2_load layout)."""
        N, L, l0, nV, nT, nS, na, nn, nD = self._sizes()
        nr = sum(2 ** l for l in range(l0, L + 1))
        r = dict(N=N, L=L, l0=l0, perm=np.zeros(N, np.int64), leaf_size=np.zeros(2 ** L, np.int64),
                 rank=np.zeros(nr, np.int64), V=np.zeros(nV, np.complex128), T=np.zeros(nT, np.complex128),
                 n_adm=np.zeros(L - l0 + 1, np.int64), adm=np.zeros(2 * na, np.int64),
                 S=np.zeros(nS, np.complex128), near=np.zeros(2 * nn, np.int64), D=np.zeros(nD, np.complex128),
                 dscale=np.zeros(N, np.float64))
        self._check(lib().h2_export(self._h, *[_ptr(r[k]) for k in
                                                ("perm", "leaf_size", "rank", "V", "T", "n_adm", "adm", "S",
                                                 "near", "D", "dscale")]), "h2_export")
        return r

    # ------------------------------------------------------------- compute
    def factorize(self, eps_fill, precision="fp64"):
        prec = {"fp64": H2_FP64, "mixed": H2_MIXED}[precision]
        self._check(lib().h2_factorize(self._h, float(eps_fill), prec), "h2_factorize")
        self.last_factorize = (float(eps_fill), precision)

    def set_chi(self, chi):
        """h2_set_chi: new contrast (N or scalar, > 0); the factors are invalidated."""
        c = np.ascontiguousarray(np.atleast_1d(np.asarray(chi, dtype=np.float64)))
        self._check(lib().h2_set_chi(self._h, _ptr(c), len(c)), "h2_set_chi")
        self.chi = np.broadcast_to(c, (self.N,)).copy()
        self.last_factorize = None

    def level_ranks(self, level):
        """(k0, kt): cluster ranks of tree level `level` before / after the Step-0
        basis update of the last factorization (h2_level_ranks)."""
        n = 2 ** level
        k0, kt = np.zeros(n, np.int32), np.zeros(n, np.int32)
        self._check(lib().h2_level_ranks(self._h, int(level), _ptr(k0), _ptr(kt), n), "h2_level_ranks")
        return k0, kt

    def invert(self):
        self._check(lib().h2_invert(self._h), "h2_invert")

    def _vec_call(self, b, out, fn):
        import torch
        is_torch = isinstance(b, torch.Tensor)
        one = b.ndim == 1
        if is_torch:
            if b.dtype != torch.complex128:
                raise TypeError("vectors must be complex128")
            bc = (b.reshape(1, -1) if one else b.T).contiguous()  # (nrhs, N) == N x nrhs column-major
            xc = torch.empty_like(bc) if out is None else out
            nrhs = bc.shape[0]
            fn(_ptr(bc), _ptr(xc), nrhs, 0)
            return xc.reshape(-1) if one else xc.T
        bh = np.asfortranarray(np.asarray(b, dtype=np.complex128).reshape(len(b), -1))
        xh = np.zeros_like(bh, order="F")
        fn(_ptr(bh), _ptr(xh), bh.shape[1], H2_HOST)
        return xh[:, 0] if one else xh

    def solve(self, b, adjoint=False, refine=False, tol=1e-6, max_iter=20, use_inverse=False, stream=None,
              allow_noconv=False):
        """x = A^{-1} b (A^{-H} b with adjoint=True); returns x (same kind as b)."""
        flags = (H2_ADJOINT if adjoint else 0) | (H2_REFINE if refine else 0) | (H2_USE_INVERSE if use_inverse else 0)
        it, res = ctypes.c_int(), ctypes.c_double()
        info = {}

        def fn(pb, px, nrhs, extra):
            st = lib().h2_solve(self._h, pb, px, nrhs, flags | extra, float(tol), int(max_iter), ctypes.byref(it),
                                ctypes.byref(res), _stream(stream))
            if not (allow_noconv and st == H2_ENOCONV):
                self._check(st, "h2_solve")
            info.update(iters=it.value, resid=res.value, status=st)

        x = self._vec_call(b, None, fn)
        self.last_solve = info
        return x

    def matvec(self, x, adjoint=False, stream=None):
        flags = H2_ADJOINT if adjoint else 0

        def fn(px, py, nrhs, extra):
            self._check(lib().h2_matvec(self._h, px, py, nrhs, flags | extra, _stream(stream)), "h2_matvec")

        return self._vec_call(x, None, fn)

    def grad_chi(self, x, mu, g=None, alpha=1.0, out=None, accumulate=False, stream=None):
        """grad[i] = alpha / chi_i * sum_c Re(x[i,c] conj(mu[i,c] - g[i,c])) on the device (h2_grad_chi).

        x, mu, g: torch CUDA complex128 of shape (N,) or (N, nrhs); g may be None.
        Returns (or fills) a float64 CUDA tensor of shape (N,)."""
        import torch

        def cm(a):
            if a is None:
                return None
            if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.complex128):
                raise TypeError("h2_grad_chi takes CUDA complex128 tensors")
            return (a.reshape(1, -1) if a.ndim == 1 else a.T).contiguous()

        xc, mc, gc = cm(x), cm(mu), cm(g)
        if mc.shape != xc.shape or (gc is not None and gc.shape != xc.shape) or xc.shape[1] != self.N:
            raise ValueError("x, mu, g must all be (N,) or (N, nrhs)")
        if out is None:
            out = torch.empty(self.N, dtype=torch.float64, device=xc.device)
        self._check(lib().h2_grad_chi(self._h, _ptr(xc), _ptr(mc), _ptr(gc), xc.shape[0], float(alpha), _ptr(out),
                                      H2_GRAD_ACCUMULATE if accumulate else 0, _stream(stream)), "h2_grad_chi")
        return out

    def set_opts(self, **kw):
        """h2_set_opts: change run-time tunables (apply_path, solve_graph,
        split_target, cluster_max, tile_policy, tensor_cores, gram_emulation,
        profile) of this
        context; tunables not given return to their defaults."""
        o = default_opts(**kw)
        self._check(lib().h2_set_opts(self._h, ctypes.byref(o)), "h2_set_opts")

    def stats(self):
        buf = ctypes.create_string_buffer(1 << 20)
        self._check(lib().h2_stats(self._h, buf, len(buf)), "h2_stats")
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().h2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _handles(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c._h.value if hasattr(c._h, "value") else c._h for c in ctxs])
    return arr


def factorize_batch(ctxs, eps_fill, precision="fp64"):
    """h2_factorize_batch: factorize several H2 contexts in shared launches."""
    prec = {"fp64": H2_FP64, "mixed": H2_MIXED}[precision]
    st = lib().h2_factorize_batch(_handles(ctxs), len(ctxs), float(eps_fill), prec)
    if st != H2_OK:
        raise H2Error(st, "h2_factorize_batch: " + lib().h2_last_error(ctxs[0]._h).decode())


def solve_batch(ctxs, bs, adjoint=False, refine=False, tol=1e-6, max_iter=20, use_inverse=False, stream=None,
                allow_noconv=False):
    """h2_solve_batch: x_q = A_q^{-1} b_q for CUDA complex128 tensors b_q of
    shape (N_q, nrhs) (same nrhs for all).  Returns (xs, info)."""
    import torch
    if len(bs) != len(ctxs):
        raise ValueError("one right-hand side per context")
    nrhs = bs[0].shape[1] if bs[0].ndim == 2 else 1
    bc, xc = [], []
    for b in bs:
        if not (isinstance(b, torch.Tensor) and b.is_cuda and b.dtype == torch.complex128):
            raise TypeError("h2_solve_batch takes CUDA complex128 tensors")
        if (b.shape[1] if b.ndim == 2 else 1) != nrhs:
            raise ValueError("all right-hand sides must have the same number of columns")
        t = (b.reshape(1, -1) if b.ndim == 1 else b.T).contiguous()
        bc.append(t)
        xc.append(torch.empty_like(t))
    flags = (H2_ADJOINT if adjoint else 0) | (H2_REFINE if refine else 0) | (H2_USE_INVERSE if use_inverse else 0)
    it, res = ctypes.c_int(), ctypes.c_double()
    barr = (ctypes.c_void_p * len(bc))(*[t.data_ptr() for t in bc])
    xarr = (ctypes.c_void_p * len(xc))(*[t.data_ptr() for t in xc])
    st = lib().h2_solve_batch(_handles(ctxs), len(ctxs), barr, xarr, nrhs, flags, float(tol), int(max_iter),
                              ctypes.byref(it), ctypes.byref(res), _stream(stream))
    if not (st == H2_OK or (allow_noconv and st == H2_ENOCONV)):
        raise H2Error(st, "h2_solve_batch: " + lib().h2_last_error(ctxs[0]._h).decode())
    xs = [(x.reshape(-1) if b.ndim == 1 else x.T) for x, b in zip(xc, bs)]
    return xs, dict(iters=it.value, resid=res.value, status=st)
