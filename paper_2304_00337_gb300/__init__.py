"""Python binding of libpbs, the GB300 photonic band-structure library.

Argument marshalling only: every computation runs in the CUDA kernels of
``libpbs.so`` behind the C ABI declared in ``include/pbs.h``.  Names follow
that header.  Device arrays are passed as raw pointers (for example
``torch.Tensor.data_ptr()`` of a contiguous ``complex128`` CUDA tensor) and a
CUDA stream handle (``torch.cuda.Stream.cuda_stream``); host arrays are NumPy.

There is no fallback: importing works without a GPU (to inspect the ABI), but
every call that needs the library raises when ``libpbs.so`` is missing or the
device is unavailable.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpbs.so")

# status codes
PBS_OK = 0
PBS_EINVAL = -1
PBS_ENOMEM = -2
PBS_ENOCONV = -3
PBS_ENUMERIC = -4
PBS_ETIMEOUT = -5
PBS_ECUDA = -6
PBS_ECANCELED = -7
# precision
PBS_FP64 = 0
PBS_MIXED = 1
PBS_START_RANDOM = 0
PBS_START_NESTED = 1
# operators
OPS = dict(A=0, M=1, A_MU_M=2, C=3, CH=4, L=5, LH=6, P_NODAL=7, PROLONG=8, RESTRICT=9, PROLONG_NODAL=10,
           RESTRICT_NODAL=11, VCYCLE_EDGE=12, VCYCLE_NODAL=13, PROJECT=14, RESIDUAL=15, LH_M=16)
for _k, _v in OPS.items():
    globals()["PBS_OP_" + _k] = _v


class PbsError(RuntimeError):
    """A non-OK status returned by the library."""

    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {strerror(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class pbs_c64(ct.Structure):
    _fields_ = [("re", ct.c_double), ("im", ct.c_double)]


class pbs_geom(ct.Structure):
    _fields_ = [("a", ct.c_double), ("b", ct.c_double), ("n", ct.c_int), ("m", ct.c_int),
                ("eps", ct.POINTER(ct.c_double))]


class pbs_opts(ct.Structure):
    _fields_ = [("nev", ct.c_int), ("block", ct.c_int), ("max_iter", ct.c_int), ("precision", ct.c_int),
                ("span", ct.c_int), ("tol", ct.c_double), ("mu", ct.c_double), ("nu_pre", ct.c_int),
                ("nu_post", ct.c_int), ("coarsest", ct.c_int), ("nodal_cycles", ct.c_int),
                ("extrap_depth", ct.c_int), ("seed", ct.c_uint64), ("kbatch", ct.c_int),
                ("start", ct.c_int)]


_lib = None


def lib() -> ct.CDLL:
    """Load ``libpbs.so`` (built in-tree by ``_build.build()``); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libpbs.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ct.CDLL(LIB_PATH)
    P = ct.c_void_p
    dp = ct.POINTER(ct.c_double)
    ip = ct.POINTER(ct.c_int)
    sig = {
        "pbs_create": (ct.c_int, [ct.POINTER(P), ct.c_int, ct.c_size_t]),
        "pbs_destroy": (ct.c_int, [P]),
        "pbs_default_opts": (None, [ct.POINTER(pbs_opts)]),
        "pbs_num_levels": (ct.c_int, [ct.c_int, ct.c_int, ct.c_int]),
        "pbs_solve_k": (ct.c_int, [P, ct.POINTER(pbs_geom), ct.POINTER(pbs_opts), dp, P, dp, dp, ip, P]),
        "pbs_solve_path": (ct.c_int, [P, ct.POINTER(pbs_geom), ct.POINTER(pbs_opts), ct.c_int, dp, dp, dp, ip]),
        "pbs_solve_path_vectors": (ct.c_int, [P, ct.POINTER(pbs_geom), ct.POINTER(pbs_opts), ct.c_int, dp, dp, dp, ip,
                                              ct.c_int, ip, P]),
        "pbs_solve_path_device": (ct.c_int, [P, ct.c_double, ct.c_double, ct.c_int, ct.c_int, P,
                                             ct.POINTER(pbs_opts), ct.c_int, P, P, P, P, P]),
        "pbs_apply": (ct.c_int, [P, ct.POINTER(pbs_geom), ct.POINTER(pbs_opts), ct.c_int, ct.c_int, dp, ct.c_int,
                                 P, P, P]),
        "pbs_gram": (ct.c_int, [P, ct.POINTER(pbs_geom), dp, ct.c_int, P, P, P, ct.c_int, P]),
        "pbs_m_householder": (ct.c_int, [P, ct.POINTER(pbs_geom), dp, ct.c_int, P, P, P, P]),
        "pbs_rayleigh_ritz": (ct.c_int, [P, ct.POINTER(pbs_geom), ct.POINTER(pbs_opts), dp, ct.c_int, P, ct.c_int,
                                         ct.c_int, dp, P, P]),
        "pbs_profile_enable": (ct.c_int, [P, ct.c_char_p]),
        "pbs_profile_read": (ct.c_int, [P, ct.c_char_p, ct.POINTER(ct.c_double), ct.POINTER(ct.c_long),
                                        ct.POINTER(ct.c_double)]),
        "pbs_launch_count": (ct.c_ulonglong, []),
        "pbs_launch_count_df": (ct.c_ulonglong, []),
        "pbs_small_rr_noalloc": (ct.c_int, [P, P, ct.c_int, ct.c_int, P, P, P, P]),
        "pbs_solve_grid": (ct.c_int, [P, ct.POINTER(pbs_geom), ct.POINTER(pbs_opts), ct.c_int, dp, dp, dp, ip]),
        "pbs_job_bytes": (ct.c_int, [ct.c_int, ct.c_int, ct.POINTER(pbs_opts), ct.c_int, ct.POINTER(ct.c_size_t)]),
        "pbs_submit": (ct.c_int, [P, ct.POINTER(pbs_geom), ct.POINTER(pbs_opts), ct.c_int, dp,
                                  ct.POINTER(ct.c_uint64)]),
        "pbs_poll": (ct.c_int, [P, ct.c_uint64, ip]),
        "pbs_fetch": (ct.c_int, [P, ct.c_uint64, dp, dp, ip, dp]),
        "pbs_cancel": (ct.c_int, [P, ct.c_uint64]),
        "pbs_job_times": (ct.c_int, [P, ct.c_uint64, dp, dp, dp]),
        "pbs_serve_slots": (ct.c_int, [P, ct.c_int]),
        "pbs_set_budget": (ct.c_int, [P, ct.c_size_t]),
        "pbs_fail_alloc_after": (ct.c_int, [P, ct.c_int]),
        "pbs_strerror": (ct.c_char_p, [ct.c_int]),
        "pbs_last_error": (ct.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def launch_count() -> int:
    """Kernels launched by the library in this process (``pbs_launch_count``)."""
    return int(lib().pbs_launch_count())


def launch_count_df() -> int:
    """Launches of double-float kernels in this process (``pbs_launch_count_df``)."""
    return int(lib().pbs_launch_count_df())


def small_rr_noalloc(gm_ptr: int, ga_ptr: int, q: int, p: int, c_ptr: int, theta_ptr: int, info_ptr: int,
                     stream=None) -> None:
    """``pbs_small_rr_noalloc``: the Rayleigh-Ritz coefficient step on device Gram matrices,
    without any device allocation (for callers that cannot call cudaMalloc)."""
    _check(lib().pbs_small_rr_noalloc(gm_ptr, ga_ptr, q, p, c_ptr, theta_ptr, info_ptr, _stream_ptr(stream)),
           "pbs_small_rr_noalloc")


def job_bytes(n: int, m: int, opts, nk: int) -> int:
    """Device bytes a path job needs (``pbs_job_bytes``, the admission estimate)."""
    o = _opts(opts)
    b = ct.c_size_t(0)
    _check(lib().pbs_job_bytes(n, m, ct.byref(o), nk, ct.byref(b)), "pbs_job_bytes")
    return int(b.value)


def strerror(status: int) -> str:
    return lib().pbs_strerror(status).decode()


def last_error() -> str:
    return lib().pbs_last_error().decode()


def _check(status: int, where: str, allow=(PBS_OK,)):
    if status not in allow:
        raise PbsError(status, where, last_error())
    return status


def default_opts(**overrides) -> pbs_opts:
    """``pbs_default_opts`` plus keyword overrides (field names of ``pbs_opts``)."""
    o = pbs_opts()
    lib().pbs_default_opts(ct.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def num_levels(n: int, m: int, coarsest: int = 4) -> int:
    return lib().pbs_num_levels(n, m, coarsest)


def _dp(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


class Geometry:
    """Cell ``a x b``, mesh ``n x m`` and cell-centre permittivity samples (shape ``(m, n)``)."""

    def __init__(self, eps, a: float = 1.0, b: float = 1.0):
        self.eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
        if self.eps.ndim != 2:
            raise ValueError("eps must have shape (m, n)")
        self.m, self.n = self.eps.shape
        self.a, self.b = float(a), float(b)
        self._g = pbs_geom(self.a, self.b, self.n, self.m, _dp(self.eps))

    @property
    def N(self) -> int:
        return self.n * self.m

    @property
    def D(self) -> int:
        return 2 * self.n * self.m

    def ref(self):
        return ct.byref(self._g)


def _opts(opts) -> pbs_opts:
    if opts is None:
        return default_opts()
    if isinstance(opts, dict):
        return default_opts(**opts)
    return opts


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


class Context:
    """Owns a ``pbs_ctx`` (device memory, resident hierarchy) on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._ptr = ct.c_void_p()
        self._jobs = {}  # job id -> (nk, nev) for sizing pbs_fetch's outputs
        _check(lib().pbs_create(ct.byref(self._ptr), device, hbm_budget_bytes), "pbs_create")

    def close(self):
        if self._ptr:
            _check(lib().pbs_destroy(self._ptr), "pbs_destroy")
            self._ptr = ct.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve_k(self, geom: Geometry, opts=None, k=(0.0, 0.0), init=None, want_vectors: bool = False,
                allow_noconv: bool = False):
        """``pbs_solve_k``; returns ``(eigvals, resid, iters, evecs or None)``.

        ``init``: complex array of shape ``(block, D)`` (row c = column c) or None.
        ``evecs``: complex array of shape ``(nev, D)``.
        """
        o = _opts(opts)
        kk = np.asarray(k, dtype=np.float64)
        ev = np.zeros(o.nev)
        rs = np.zeros(o.nev)
        it = ct.c_int(0)
        init_p = None
        if init is not None:
            init_arr = np.ascontiguousarray(np.asarray(init, dtype=np.complex128))
            if init_arr.shape != (o.block, geom.D):
                raise ValueError("init must have shape (block, D)")
            init_p = init_arr.ctypes.data
        vec = np.zeros((o.nev, geom.D), np.complex128) if want_vectors else None
        st = lib().pbs_solve_k(self._ptr, geom.ref(), ct.byref(o), _dp(kk), init_p, _dp(ev), _dp(rs), ct.byref(it),
                               vec.ctypes.data if vec is not None else None)
        _check(st, "pbs_solve_k", (PBS_OK, PBS_ENOCONV) if allow_noconv else (PBS_OK,))
        return ev, rs, it.value, vec

    def solve_path(self, geom: Geometry, opts, ks, allow_noconv: bool = False):
        """``pbs_solve_path`` over ``ks`` (shape ``(nk, 2)``); returns ``(eigvals, resid, iters)``."""
        o = _opts(opts)
        kk = np.ascontiguousarray(np.asarray(ks, dtype=np.float64).reshape(-1, 2))
        nk = kk.shape[0]
        ev = np.zeros((nk, o.nev))
        rs = np.zeros((nk, o.nev))
        it = np.zeros(nk, dtype=np.int32)
        st = lib().pbs_solve_path(self._ptr, geom.ref(), ct.byref(o), nk, _dp(kk), _dp(ev), _dp(rs),
                                  it.ctypes.data_as(ct.POINTER(ct.c_int)))
        _check(st, "pbs_solve_path", (PBS_OK, PBS_ENOCONV) if allow_noconv else (PBS_OK,))
        return ev, rs, it

    def solve_path_vectors(self, geom: Geometry, opts, ks, sel, allow_noconv: bool = False):
        """``pbs_solve_path_vectors``: ``solve_path`` plus the M-normalised eigenvectors of the
        Bloch vectors ``sel``; returns ``(eigvals, resid, iters, vecs)`` with ``vecs`` of shape
        ``(len(sel), nev, D)`` (row ``j`` = eigenvector of band ``j``)."""
        o = _opts(opts)
        kk = np.ascontiguousarray(np.asarray(ks, dtype=np.float64).reshape(-1, 2))
        nk = kk.shape[0]
        sl = np.ascontiguousarray(np.asarray(sel, dtype=np.int32).reshape(-1))
        ev = np.zeros((nk, o.nev))
        rs = np.zeros((nk, o.nev))
        it = np.zeros(nk, dtype=np.int32)
        vecs = np.zeros((sl.size, o.nev, geom.D), dtype=np.complex128)
        st = lib().pbs_solve_path_vectors(self._ptr, geom.ref(), ct.byref(o), nk, _dp(kk), _dp(ev), _dp(rs),
                                          it.ctypes.data_as(ct.POINTER(ct.c_int)), int(sl.size),
                                          sl.ctypes.data_as(ct.POINTER(ct.c_int)), vecs.ctypes.data)
        _check(st, "pbs_solve_path_vectors", (PBS_OK, PBS_ENOCONV) if allow_noconv else (PBS_OK,))
        return ev, rs, it, vecs

    def solve_grid(self, geom: Geometry, opts, kappa: int, allow_noconv: bool = False):
        """``pbs_solve_grid``: the kappa x kappa sample with the paper's extrapolation schedule;
        returns ``(ks, eigvals, resid, iters)`` indexed ``j * kappa + i``."""
        o = _opts(opts)
        nk = kappa * kappa
        ks = np.zeros((nk, 2))
        ev = np.zeros((nk, o.nev))
        rs = np.zeros((nk, o.nev))
        it = np.zeros(nk, dtype=np.int32)
        st = lib().pbs_solve_grid(self._ptr, geom.ref(), ct.byref(o), kappa, _dp(ks), _dp(ev), _dp(rs),
                                  it.ctypes.data_as(ct.POINTER(ct.c_int)))
        _check(st, "pbs_solve_grid", (PBS_OK, PBS_ENOCONV) if allow_noconv else (PBS_OK,))
        return ks, ev, rs, it

    def submit(self, geom: Geometry, opts, ks) -> int:
        """``pbs_submit``: queue a path job; returns its id at once."""
        o = _opts(opts)
        kk = np.ascontiguousarray(np.asarray(ks, dtype=np.float64).reshape(-1, 2))
        jid = ct.c_uint64(0)
        _check(lib().pbs_submit(self._ptr, geom.ref(), ct.byref(o), kk.shape[0], _dp(kk), ct.byref(jid)),
               "pbs_submit")
        self._jobs[int(jid.value)] = (kk.shape[0], o.nev)
        return int(jid.value)

    def poll(self, job: int) -> bool:
        """``pbs_poll``: True once the job has finished."""
        d = ct.c_int(0)
        _check(lib().pbs_poll(self._ptr, job, ct.byref(d)), "pbs_poll")
        return bool(d.value)

    def fetch(self, job: int, allow_noconv: bool = False):
        """``pbs_fetch``: wait for the job; returns ``(eigvals, resid, iters, latency_s)``."""
        nk, nev = self._jobs.pop(job, (0, 0))
        ev = np.zeros((nk, nev))
        rs = np.zeros((nk, nev))
        it = np.zeros(nk, dtype=np.int32)
        lat = ct.c_double(0.0)
        st = lib().pbs_fetch(self._ptr, job, _dp(ev), _dp(rs), it.ctypes.data_as(ct.POINTER(ct.c_int)),
                             ct.byref(lat))
        _check(st, "pbs_fetch", (PBS_OK, PBS_ENOCONV) if allow_noconv else (PBS_OK,))
        return ev, rs, it, lat.value

    def cancel(self, job: int) -> None:
        """``pbs_cancel``: drop a queued job or stop a running one at its next iteration."""
        _check(lib().pbs_cancel(self._ptr, job), "pbs_cancel")

    def job_times(self, job: int):
        """``pbs_job_times``: (submitted, started, finished) in seconds since the context's creation."""
        a, b, c = ct.c_double(), ct.c_double(), ct.c_double()
        _check(lib().pbs_job_times(self._ptr, job, ct.byref(a), ct.byref(b), ct.byref(c)), "pbs_job_times")
        return a.value, b.value, c.value

    def serve_slots(self, slots: int) -> None:
        """``pbs_serve_slots``: number of concurrent serving slots (before the first submission)."""
        _check(lib().pbs_serve_slots(self._ptr, slots), "pbs_serve_slots")

    def set_budget(self, hbm_budget_bytes: int) -> None:
        """``pbs_set_budget``: change the byte budget of the context's own allocations."""
        _check(lib().pbs_set_budget(self._ptr, hbm_budget_bytes), "pbs_set_budget")

    def fail_alloc_after(self, count: int) -> None:
        """``pbs_fail_alloc_after``: make the count-th device allocation from now fail (tests)."""
        _check(lib().pbs_fail_alloc_after(self._ptr, count), "pbs_fail_alloc_after")

    def solve_path_device(self, a, b, n, m, d_eps: int, opts, nk: int, d_ks: int, d_eigvals: int, d_resid: int,
                          d_iters: int, stream=None, allow_noconv: bool = False):
        """``pbs_solve_path_device`` with raw device pointers."""
        o = _opts(opts)
        st = lib().pbs_solve_path_device(self._ptr, a, b, n, m, d_eps, ct.byref(o), nk, d_ks, d_eigvals, d_resid,
                                         d_iters, _stream_ptr(stream))
        _check(st, "pbs_solve_path_device", (PBS_OK, PBS_ENOCONV) if allow_noconv else (PBS_OK,))
        return st

    def apply(self, geom: Geometry, op, x_ptr: int, y_ptr: int, ncols: int, k=(0.0, 0.0), level: int = 0,
              opts=None, stream=None):
        """``pbs_apply`` on device arrays (interleaved complex128)."""
        o = _opts(opts)
        opc = OPS[op] if isinstance(op, str) else int(op)
        kk = np.asarray(k, dtype=np.float64)
        _check(lib().pbs_apply(self._ptr, geom.ref(), ct.byref(o), opc, level, _dp(kk), ncols, x_ptr, y_ptr,
                               _stream_ptr(stream)), f"pbs_apply({op})")

    def gram(self, geom: Geometry, k, q: int, s_ptr: int, gm_ptr: int, ga_ptr: int, stream=None,
             precision: int = PBS_FP64):
        kk = np.asarray(k, dtype=np.float64)
        _check(lib().pbs_gram(self._ptr, geom.ref(), _dp(kk), q, s_ptr, gm_ptr, ga_ptr, precision,
                              _stream_ptr(stream)), "pbs_gram")

    def m_householder(self, geom: Geometry, k, q: int, s_ptr: int, e_ptr: int, r_ptr: int, stream=None):
        """Generalised Householder factorisation ``S = E R`` with ``E^* M E = I`` (``pbs_m_householder``).

        ``s_ptr``, ``e_ptr``: device ``D x q`` column-major complex128; ``r_ptr``: device ``q x q``.
        """
        kk = np.asarray(k, dtype=np.float64)
        _check(lib().pbs_m_householder(self._ptr, geom.ref(), _dp(kk), q, s_ptr, e_ptr, r_ptr, _stream_ptr(stream)),
               "pbs_m_householder")

    def profile_enable(self, classes: str | None):
        """Time kernel classes with CUDA events on the library's stream (``pbs_profile_enable``)."""
        _check(lib().pbs_profile_enable(self._ptr, (classes or "").encode()), "pbs_profile_enable")

    def profile_read(self, kernel_class: str):
        """``(total_ms, launches, work)`` of one timed kernel class (``pbs_profile_read``)."""
        ms = ct.c_double(0.0)
        n = ct.c_long(0)
        w = ct.c_double(0.0)
        _check(lib().pbs_profile_read(self._ptr, kernel_class.encode(), ct.byref(ms), ct.byref(n), ct.byref(w)),
               "pbs_profile_read")
        return ms.value, n.value, w.value

    def rayleigh_ritz(self, geom: Geometry, opts, k, q: int, s_ptr: int, p: int, project: bool, x_ptr: int,
                      stream=None):
        o = _opts(opts)
        kk = np.asarray(k, dtype=np.float64)
        theta = np.zeros(p)
        _check(lib().pbs_rayleigh_ritz(self._ptr, geom.ref(), ct.byref(o), _dp(kk), q, s_ptr, p, int(bool(project)),
                                       _dp(theta), x_ptr, _stream_ptr(stream)), "pbs_rayleigh_ritz")
        return theta


def abi_symbols_from_header(path: str | None = None) -> list[str]:
    """Names of the functions ``include/pbs.h`` declares (for export checks)."""
    import re
    path = path or os.path.join(os.path.dirname(_PKG), "include", "pbs.h")
    txt = open(path).read()
    return sorted(set(re.findall(r"PBS_API\s+[\w\s\*]*?\b(pbs_\w+)\s*\(", txt)))
