"""GB300-native Newton-multigrid solver for marble sulfation (arXiv:1902.07029).

Thin ctypes binding of the C ABI in ``include/sulfmg.h`` (and the stage-level
entry points of ``include/sulfmg_debug.h``).  This module only marshals
arguments: every stage of the method runs in the CUDA kernels of
``libsulfmg.so``.  There is no CPU fallback -- if the library is missing or no
GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB_PATH, build  # noqa: F401

OK, EINVAL, ENOMEM, ENOTCONV, EGEOM, EDEVICE = 0, -1, -2, -3, -4, -5


class SulfModel(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("a", "d", "m_s", "m_c", "alpha", "beta", "s_ext", "s0", "c0")]


class SulfSolver(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("cycle", ctypes.c_int), ("max_newton", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("ghost_sweeps", ctypes.c_int), ("newton_tol", ctypes.c_double),
                ("lin_rtol", ctypes.c_double), ("tau_s", ctypes.c_double), ("precision", ctypes.c_int),
                ("smoother", ctypes.c_int), ("graphs", ctypes.c_int), ("fuse_below", ctypes.c_int),
                ("pdl", ctypes.c_int), ("ghost_compose", ctypes.c_int), ("relax_occupancy", ctypes.c_int),
                ("relax_matrix_free", ctypes.c_int)]


class SulfStats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("newton_last", ctypes.c_int), ("cycles_last", ctypes.c_int),
                ("newton_total", ctypes.c_longlong), ("cycles_total", ctypes.c_longlong),
                ("steps_total", ctypes.c_longlong), ("last_rho", ctypes.c_double), ("last_fnorm", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("levels", ctypes.c_int), ("n_inside", ctypes.c_longlong),
                ("n_ghost", ctypes.c_longlong), ("ghost_rows", ctypes.c_int * 3),
                ("device_bytes", ctypes.c_ulonglong), ("loop_graph", ctypes.c_int)]


class SulfJob(ctypes.Structure):
    _fields_ = [("levelset", ctypes.POINTER(ctypes.c_double)), ("dim", ctypes.c_int), ("N", ctypes.c_int),
                ("coarsest_N", ctypes.c_int), ("box_lo", ctypes.c_double), ("box_hi", ctypes.c_double),
                ("model", SulfModel), ("solver", SulfSolver), ("dt", ctypes.c_double), ("nsteps", ctypes.c_int)]


class SulfJobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("estimate_bytes", ctypes.c_ulonglong),
                ("device_bytes", ctypes.c_ulonglong), ("newton", ctypes.c_longlong), ("cycles", ctypes.c_longlong)]


class SulfTuneResult(ctypes.Structure):
    _fields_ = [("fuse_below", ctypes.c_int), ("ghost_compose", ctypes.c_int), ("pdl", ctypes.c_int),
                ("relax_occupancy", ctypes.c_int), ("relax_matrix_free", ctypes.c_int),
                ("ms_per_cycle", ctypes.c_double), ("ms_per_cycle_default", ctypes.c_double),
                ("candidates", ctypes.c_int), ("cached", ctypes.c_int)]


class SulfServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong), ("queued", ctypes.c_longlong),
                ("running", ctypes.c_longlong), ("max_running", ctypes.c_longlong), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("jobs_per_s", ctypes.c_double), ("budget_bytes", ctypes.c_ulonglong),
                ("peak_reserved_bytes", ctypes.c_ulonglong)]


_lib = None
P = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i8p = ctypes.POINTER(ctypes.c_int8)
_i64p = ctypes.POINTER(ctypes.c_int64)

_SIGS = {
    "sulf_create_domain": (ctypes.c_int, [_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)]),
    "sulf_set_model": (ctypes.c_int, [P, ctypes.POINTER(SulfModel)]),
    "sulf_set_solver": (ctypes.c_int, [P, ctypes.POINTER(SulfSolver)]),
    "sulf_set_stream": (ctypes.c_int, [P, P]),
    "sulf_step": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_int]),
    "sulf_get_state": (ctypes.c_int, [P, _dp, _dp, _i8p]),
    "sulf_get_state_device": (ctypes.c_int, [P, P, P]),
    "sulf_set_state": (ctypes.c_int, [P, _dp, _dp, ctypes.c_double]),
    "sulf_set_state_device": (ctypes.c_int, [P, P, P, ctypes.c_double]),
    "sulf_get_stats": (ctypes.c_int, [P, ctypes.POINTER(SulfStats)]),
    "sulf_reinit_levelset": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]),
    "sulf_levelset_from_mask": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint8), ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _dp]),
    "sulf_set_state_extrapolated": (ctypes.c_int, [P, _dp, _dp, ctypes.c_double]),
    "sulf_set_bc": (ctypes.c_int, [P, ctypes.c_int]),
    "sulf_dbg_level_rows": (ctypes.c_int, [P, ctypes.c_int, _dp, _dp]),
    "sulf_set_sources": (ctypes.c_int, [P, _dp, _dp, _dp, _dp]),
    "sulf_set_ghost_values": (ctypes.c_int, [P, _dp]),
    "sulf_set_profiling": (ctypes.c_int, [P, ctypes.c_int]),
    "sulf_kernel_time": (ctypes.c_int, [P, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "sulf_newton_residual_noalloc": (ctypes.c_int, [P, ctypes.c_double, P, P, P, P]),
    "sulf_batch_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)]),
    "sulf_batch_step": (ctypes.c_int, [P, _dp, ctypes.POINTER(ctypes.c_int)]),
    "sulf_batch_status": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int)]),
    "sulf_batch_set_lockstep": (ctypes.c_int, [P, ctypes.c_int]),
    "sulf_batch_autotune": (ctypes.c_int, [P, _dp, ctypes.POINTER(SulfTuneResult)]),
    "sulf_autotune": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(SulfTuneResult)]),
    "sulf_batch_destroy": (None, [P]),
    "sulf_estimate_device_bytes": (ctypes.c_ulonglong, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "sulf_server_create": (ctypes.c_int, [ctypes.c_ulonglong, ctypes.c_int, ctypes.POINTER(P)]),
    "sulf_server_submit": (ctypes.c_int, [P, ctypes.POINTER(SulfJob), ctypes.POINTER(ctypes.c_longlong)]),
    "sulf_server_poll": (ctypes.c_int, [P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]),
    "sulf_server_wait": (ctypes.c_int, [P, ctypes.c_longlong, _dp, _dp, ctypes.POINTER(SulfJobResult)]),
    "sulf_server_get_stats": (ctypes.c_int, [P, ctypes.POINTER(SulfServerStats)]),
    "sulf_server_destroy": (None, [P]),
    "sulf_destroy": (None, [P]),
    "sulf_last_error": (ctypes.c_char_p, []),
    "sulf_dbg_level_info": (ctypes.c_int, [P, ctypes.c_int, _i64p]),
    "sulf_dbg_level_type": (ctypes.c_int, [P, ctypes.c_int, _i8p]),
    "sulf_dbg_level_ghosts": (ctypes.c_int, [P, ctypes.c_int, _i64p, _i8p, _i8p, _dp, _dp]),
    "sulf_dbg_eval_F": (ctypes.c_int, [P, ctypes.c_double, _dp, _dp, _dp]),
    "sulf_dbg_apply_J": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]),
    "sulf_dbg_smooth": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int]),
    "sulf_dbg_restrict": (ctypes.c_int, [P, ctypes.c_int, _dp, _dp]),
    "sulf_dbg_prolong": (ctypes.c_int, [P, ctypes.c_int, _dp, _dp]),
    "sulf_dbg_inject": (ctypes.c_int, [P, _dp, ctypes.c_int, _dp]),
    "sulf_dbg_cycles": (ctypes.c_int, [P, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int, _dp]),
    "sulf_dbg_coarsest_solve": (ctypes.c_int, [P, ctypes.c_double, _dp, _dp, _dp]),
}


def load(path: str | None = None):
    """Load libsulfmg.so (built in-tree by ``build()``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libsulfmg.so not found at {path}: run paper_1902_07029_gb300.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class SulfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sulfmg error {code}: {msg}")
        self.code = code


def _d(a):
    return a.ctypes.data_as(_dp)


def _chk(lib, rc):
    if rc != OK:
        raise SulfError(rc, lib.sulf_last_error().decode())


def default_solver(**kw) -> SulfSolver:
    s = SulfSolver(nu1=2, nu2=2, cycle=1, max_newton=20, max_cycles=30, ghost_sweeps=4, newton_tol=1e-10,
                   lin_rtol=1e-10, tau_s=0.9, precision=0, smoother=0, graphs=1, fuse_below=-1, pdl=1,
                   ghost_compose=1, relax_occupancy=0, relax_matrix_free=1)
    for k, v in kw.items():
        setattr(s, k, v)
    return s


def reinit_levelset(phi, dim, N, h, steps):
    """Reinitialization toward the signed distance (Sec. 2), on the GPU."""
    lib = load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    if phi.size != (N + 1) ** dim:
        raise ValueError("phi must hold (N+1)^dim values")
    out = np.zeros_like(phi)
    _chk(lib, lib.sulf_reinit_levelset(_d(phi), dim, N, float(h), int(steps), _d(out)))
    return out


def levelset_from_mask(mask, dim, N, steps):
    """Provisional level set of a binary mask (Sec. 2), on the GPU."""
    lib = load()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.size != (N + 1) ** dim:
        raise ValueError("mask must hold (N+1)^dim values")
    out = np.zeros(m.shape, dtype=np.float64)
    _chk(lib, lib.sulf_levelset_from_mask(m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), dim, N, int(steps),
                                          _d(out)))
    return out


class Domain:
    """A level-set domain resident on the GPU (one ``sulf_handle``)."""

    def __init__(self, levelset, dim, box, N, coarsest_N=8):
        self.lib = load()
        phi = np.ascontiguousarray(levelset, dtype=np.float64)
        if phi.size != (N + 1) ** dim:
            raise ValueError("levelset must hold (N+1)^dim values")
        b = np.asarray(box, dtype=np.float64)
        h = P()
        _chk(self.lib, self.lib.sulf_create_domain(_d(phi), dim, _d(b), N, coarsest_N, ctypes.byref(h)))
        self.h = h
        self.dim, self.N = dim, N
        self.shape = (N + 1,) * dim
        self.nn = (N + 1) ** dim

    def close(self):
        if getattr(self, "h", None):
            self.lib.sulf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_model(self, params):
        m = SulfModel(*[float(v) for v in params])
        _chk(self.lib, self.lib.sulf_set_model(self.h, ctypes.byref(m)))

    def set_solver(self, **kw):
        s = default_solver(**kw)
        _chk(self.lib, self.lib.sulf_set_solver(self.h, ctypes.byref(s)))

    def set_stream(self, stream_handle: int | None):
        _chk(self.lib, self.lib.sulf_set_stream(self.h, P(stream_handle) if stream_handle else None))

    def step(self, dt, nsteps=1):
        _chk(self.lib, self.lib.sulf_step(self.h, dt, nsteps))

    def get_state(self):
        s = np.zeros(self.nn)
        c = np.zeros(self.nn)
        t = np.zeros(self.nn, dtype=np.int8)
        _chk(self.lib, self.lib.sulf_get_state(self.h, _d(s), _d(c), t.ctypes.data_as(_i8p)))
        return s.reshape(self.shape), c.reshape(self.shape), t.reshape(self.shape)

    def get_state_into(self, s, c):
        """Host arrays (e.g. pinned torch tensors' numpy views) of nn doubles."""
        _chk(self.lib, self.lib.sulf_get_state(self.h, _d(s), _d(c), None))

    def get_state_device(self, s_ptr: int, c_ptr: int):
        _chk(self.lib, self.lib.sulf_get_state_device(self.h, P(s_ptr), P(c_ptr)))

    def set_state(self, s, c, t=0.0):
        s = np.ascontiguousarray(s, dtype=np.float64).ravel()
        c = np.ascontiguousarray(c, dtype=np.float64).ravel()
        _chk(self.lib, self.lib.sulf_set_state(self.h, _d(s), _d(c), t))

    def set_state_extrapolated(self, s, c, t=0.0):
        """Set the state from its inside values; the ghost values are
        extrapolated (second order) from them."""
        s = np.ascontiguousarray(s, dtype=np.float64).ravel()
        c = np.ascontiguousarray(c, dtype=np.float64).ravel()
        _chk(self.lib, self.lib.sulf_set_state_extrapolated(self.h, _d(s), _d(c), t))

    def set_state_device(self, s_ptr: int, c_ptr: int, t=0.0):
        _chk(self.lib, self.lib.sulf_set_state_device(self.h, P(s_ptr), P(c_ptr), t))

    def stats(self):
        st = SulfStats()
        _chk(self.lib, self.lib.sulf_get_stats(self.h, ctypes.byref(st)))
        return {f[0]: (list(getattr(st, f[0])) if f[0] == "ghost_rows" else getattr(st, f[0])) for f in st._fields_}

    def newton_residual_noalloc(self, dt, W_ptr: int, Wn_ptr: int, F_ptr: int, fnorm_ptr: int):
        """F(W; W^n) and |F|_inf on caller-owned device buffers (device
        pointers as ints); queued on the handle's stream, no allocation."""
        _chk(self.lib, self.lib.sulf_newton_residual_noalloc(self.h, dt, P(W_ptr), P(Wn_ptr), P(F_ptr),
                                                             P(fnorm_ptr)))

    def autotune(self, dt, use_cache=True):
        """Time the speed-only solver controls on this domain's Newton system
        and keep the fastest (sulf_autotune); returns the result as a dict."""
        r = SulfTuneResult()
        _chk(self.lib, self.lib.sulf_autotune(self.h, dt, int(bool(use_cache)), ctypes.byref(r)))
        return {f[0]: getattr(r, f[0]) for f in r._fields_}

    def set_bc(self, bc):
        """0: Dirichlet s = s_b (Eq. BCs); 1: Neumann ds/dn = s_b (Eq. BCsN)."""
        _chk(self.lib, self.lib.sulf_set_bc(self.h, int(bc)))

    def level_rows(self, l):
        """Member weights of every ghost row (ng x 3^dim) and the unit normal of
        the interpolated level set at each boundary point (ng x dim)."""
        ng = self.level_info(l)["ng"]
        d = self.dim
        K = 9 if d == 2 else 27
        wk = np.zeros(max(ng, 1) * K)
        nt = np.zeros(max(ng, 1) * d)
        _chk(self.lib, self.lib.sulf_dbg_level_rows(self.h, l, _d(wk), _d(nt)))
        return wk[:ng * K].reshape(ng, K), nt[:ng * d].reshape(ng, d)

    def set_sources(self, f1_old=None, f1_new=None, f2_old=None, f2_new=None):
        """Manufactured source terms at t_n and t_{n+1} (box arrays), or none."""
        if f1_old is None:
            _chk(self.lib, self.lib.sulf_set_sources(self.h, None, None, None, None))
            return
        arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (f1_old, f1_new, f2_old, f2_new)]
        if any(a.size != self.nn for a in arrs):
            raise ValueError("source arrays must hold (N+1)^dim values")
        _chk(self.lib, self.lib.sulf_set_sources(self.h, *[_d(a) for a in arrs]))

    def set_ghost_values(self, sb=None):
        """Dirichlet values per finest-level ghost (ghost order), or None for s_ext."""
        if sb is None:
            _chk(self.lib, self.lib.sulf_set_ghost_values(self.h, None))
            return
        sb = np.ascontiguousarray(sb, dtype=np.float64).ravel()
        _chk(self.lib, self.lib.sulf_set_ghost_values(self.h, _d(sb)))

    def set_profiling(self, on):
        """0/False off; 1/True the first finest-level sweep of every cycle; 2
        every finest-level sweep."""
        _chk(self.lib, self.lib.sulf_set_profiling(self.h, int(on)))

    def kernel_time(self):
        ms = ctypes.c_double(0)
        n = ctypes.c_longlong(0)
        _chk(self.lib, self.lib.sulf_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # ---- stage-level entry points (interleaved (s,c) arrays) ----
    def level_info(self, l):
        info = np.zeros(11, dtype=np.int64)
        _chk(self.lib, self.lib.sulf_dbg_level_info(self.h, l, info.ctypes.data_as(_i64p)))
        return dict(N=int(info[0]), n=int(info[1]), ng=int(info[2]), nb=int(info[3]), nact=int(info[4]),
                    nin=int(info[5]), kinds=(int(info[6]), int(info[7]), int(info[8])),
                    ghost_map_entries=int(info[9]), ghost_map_passes=int(info[10]))

    def level_type(self, l):
        n = self.level_info(l)["n"]
        t = np.zeros(n ** self.dim, dtype=np.int8)
        _chk(self.lib, self.lib.sulf_dbg_level_type(self.h, l, t.ctypes.data_as(_i8p)))
        return t

    def level_ghosts(self, l):
        ng = self.level_info(l)["ng"]
        d = self.dim
        idx = np.zeros(max(ng, 1), dtype=np.int64)
        kind = np.zeros(max(ng, 1), dtype=np.int8)
        m = np.zeros(max(ng, 1) * d, dtype=np.int8)
        w = np.zeros(max(ng, 1) * d * 3)
        B = np.zeros(max(ng, 1) * d)
        _chk(self.lib, self.lib.sulf_dbg_level_ghosts(self.h, l, idx.ctypes.data_as(_i64p), kind.ctypes.data_as(_i8p),
                                                      m.ctypes.data_as(_i8p), _d(w), _d(B)))
        return dict(idx=idx[:ng], kind=kind[:ng], m=m[:ng * d].reshape(ng, d), w=w[:ng * d * 3].reshape(ng, d, 3),
                    B=B[:ng * d].reshape(ng, d))

    def eval_F(self, dt, W, Wn):
        W = np.ascontiguousarray(W, dtype=np.float64)
        Wn = np.ascontiguousarray(Wn, dtype=np.float64)
        F = np.zeros(2 * self.nn)
        _chk(self.lib, self.lib.sulf_dbg_eval_F(self.h, dt, _d(W), _d(Wn), _d(F)))
        return F

    def apply_J(self, l, dt, Wc, x):
        Wc = np.ascontiguousarray(Wc, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        _chk(self.lib, self.lib.sulf_dbg_apply_J(self.h, l, dt, _d(Wc), _d(x), _d(out)))
        return out

    def smooth(self, l, dt, Wc, rhs, x, sweeps=1):
        x = np.array(x, dtype=np.float64)
        Wc = np.ascontiguousarray(Wc, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        _chk(self.lib, self.lib.sulf_dbg_smooth(self.h, l, dt, _d(Wc), _d(rhs), _d(x), sweeps))
        return x

    def restrict(self, l, res):
        res = np.array(res, dtype=np.float64)
        nc = self.level_info(l + 1)["n"] ** self.dim
        out = np.zeros(2 * nc)
        _chk(self.lib, self.lib.sulf_dbg_restrict(self.h, l, _d(res), _d(out)))
        return out, res

    def prolong(self, l, xc, xf):
        xc = np.ascontiguousarray(xc, dtype=np.float64)
        xf = np.array(xf, dtype=np.float64)
        _chk(self.lib, self.lib.sulf_dbg_prolong(self.h, l, _d(xc), _d(xf)))
        return xf

    def inject(self, Wc0, l):
        Wc0 = np.ascontiguousarray(Wc0, dtype=np.float64)
        out = np.zeros(2 * self.level_info(l)["n"] ** self.dim)
        _chk(self.lib, self.lib.sulf_dbg_inject(self.h, _d(Wc0), l, _d(out)))
        return out

    def coarsest_solve(self, dt, Wc0, rhs_c):
        Wc0 = np.ascontiguousarray(Wc0, dtype=np.float64)
        rhs_c = np.ascontiguousarray(rhs_c, dtype=np.float64)
        x = np.zeros_like(rhs_c)
        _chk(self.lib, self.lib.sulf_dbg_coarsest_solve(self.h, dt, _d(Wc0), _d(rhs_c), _d(x)))
        return x

    def cycles(self, dt, Wc0, rhs, ncycles):
        Wc0 = np.ascontiguousarray(Wc0, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.zeros_like(rhs)
        rn = np.zeros(ncycles)
        _chk(self.lib, self.lib.sulf_dbg_cycles(self.h, dt, _d(Wc0), _d(rhs), _d(x), ncycles, _d(rn)))
        return x, rn


class Batch:
    """Many domains advanced together (each keeps its own state and results)."""

    def __init__(self, domains, nstreams=8, lockstep=False):
        self.lib = load()
        self.domains = list(domains)
        arr = (P * len(self.domains))(*[d.h for d in self.domains])
        b = P()
        _chk(self.lib, self.lib.sulf_batch_create(arr, len(self.domains), nstreams, ctypes.byref(b)))
        self.b = b
        if lockstep:
            self.set_lockstep(lockstep)

    def set_lockstep(self, mode):
        """sulf_batch_set_lockstep: same-class instances step in lock step
        (False/0 off, True/1 chunks of at most 32, m >= 2 chunks of at most m)"""
        _chk(self.lib, self.lib.sulf_batch_set_lockstep(self.b, int(mode)))

    def step(self, dt, nsteps):
        n = len(self.domains)
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        ns = np.ascontiguousarray(np.broadcast_to(np.asarray(nsteps, dtype=np.int32), (n,)))
        _chk(self.lib, self.lib.sulf_batch_step(self.b, _d(dts), ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))

    def autotune(self, dt):
        """sulf_batch_autotune: one timing per problem class; per-instance results"""
        n = len(self.domains)
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        res = (SulfTuneResult * n)()
        _chk(self.lib, self.lib.sulf_batch_autotune(self.b, _d(dts), res))
        return [{f[0]: getattr(r, f[0]) for f in r._fields_} for r in res]

    def status(self):
        st = np.zeros(len(self.domains), dtype=np.int32)
        _chk(self.lib, self.lib.sulf_batch_status(self.b, st.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return st

    def close(self):
        if getattr(self, "b", None):
            self.lib.sulf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_device_bytes(dim, N, coarsest_N=8, precision=0):
    return int(load().sulf_estimate_device_bytes(dim, N, coarsest_N, precision))


class Server:
    """Continuous batching of time-stepping jobs under a device-memory budget."""

    def __init__(self, budget_bytes, nworkers=4):
        self.lib = load()
        s = P()
        _chk(self.lib, self.lib.sulf_server_create(int(budget_bytes), nworkers, ctypes.byref(s)))
        self.s = s
        self._shape = {}

    def submit(self, levelset, dim, N, model, dt, nsteps, box=(-1.0, 1.0), coarsest_N=8, **solver):
        phi = np.ascontiguousarray(levelset, dtype=np.float64)
        job = SulfJob(levelset=_d(phi), dim=dim, N=N, coarsest_N=coarsest_N, box_lo=box[0], box_hi=box[1],
                      model=SulfModel(*[float(v) for v in model]), solver=default_solver(**solver), dt=dt,
                      nsteps=nsteps)
        jid = ctypes.c_longlong(0)
        _chk(self.lib, self.lib.sulf_server_submit(self.s, ctypes.byref(job), ctypes.byref(jid)))
        self._shape[jid.value] = phi.shape
        return jid.value

    def done(self, jid):
        d = ctypes.c_int(0)
        _chk(self.lib, self.lib.sulf_server_poll(self.s, jid, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, jid):
        """(s, c, result dict); raises SulfError if the job failed."""
        shape = self._shape.pop(jid)
        nn = int(np.prod(shape))
        s = np.zeros(nn)
        c = np.zeros(nn)
        r = SulfJobResult()
        rc = self.lib.sulf_server_wait(self.s, jid, _d(s), _d(c), ctypes.byref(r))
        res = {f[0]: getattr(r, f[0]) for f in r._fields_}
        if rc != OK:
            err = SulfError(rc, self.lib.sulf_last_error().decode())
            err.result = res
            raise err
        return s.reshape(shape), c.reshape(shape), res

    def stats(self):
        st = SulfServerStats()
        _chk(self.lib, self.lib.sulf_server_get_stats(self.s, ctypes.byref(st)))
        return {f[0]: getattr(st, f[0]) for f in st._fields_}

    def close(self):
        if getattr(self, "s", None):
            self.lib.sulf_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
