"""CPU oracle for the sulfation Newton-multigrid step (test infrastructure).

A ctypes wrapper around ``sulf_oracle.c``: plain single-threaded FP64 C that
restates Sec. 3 of arXiv:1902.07029.  It is used only by the tests, by the
package smoke check and by the benchmark's CPU-baseline and reference legs, to
check and time the CUDA library; the product path never loads it.  It shares no
code with the CUDA implementation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sulf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOMEM, ENOTCONV, EGEOM = 0, -1, -2, -3, -4

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_long)
    bp = ctypes.POINTER(ctypes.c_byte)
    ip = ctypes.POINTER(ctypes.c_int)
    sigs = {
        "oracle_create": (P, [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, ip]),
        "oracle_destroy": (None, [P]),
        "oracle_last_error": (ctypes.c_char_p, []),
        "oracle_set_model": (ctypes.c_int, [P, dp]),
        "oracle_set_solver": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int]),
        "oracle_step": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_int]),
        "oracle_get_state": (ctypes.c_int, [P, dp, dp, bp]),
        "oracle_set_state": (ctypes.c_int, [P, dp, dp, ctypes.c_double]),
        "oracle_get_stats": (ctypes.c_int, [P, lp, dp]),
        "oracle_get_rho": (ctypes.c_int, [P, dp, bp, ctypes.c_int]),
        "oracle_clear_rho": (None, [P]),
        "oracle_num_levels": (ctypes.c_int, [P]),
        "oracle_level_info": (ctypes.c_int, [P, ctypes.c_int, lp]),
        "oracle_level_type": (ctypes.c_int, [P, ctypes.c_int, bp]),
        "oracle_level_phi": (ctypes.c_int, [P, ctypes.c_int, dp]),
        "oracle_level_ghosts": (ctypes.c_int, [P, ctypes.c_int, lp, bp, bp, dp, dp]),
        "oracle_level_band": (ctypes.c_int, [P, ctypes.c_int, lp, lp, dp]),
        "oracle_set_ghost_sb": (ctypes.c_int, [P, dp]),
        "oracle_set_sources": (ctypes.c_int, [P, dp, dp, dp, dp]),
        "oracle_set_bc": (ctypes.c_int, [P, ctypes.c_int]),
        "oracle_reinit": (ctypes.c_int, [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp]),
        "oracle_mask_levelset": (ctypes.c_int, [bp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]),
        "oracle_extrapolate": (ctypes.c_int, [dp, bp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp]),
        "oracle_level_rows": (ctypes.c_int, [P, ctypes.c_int, dp, dp]),
        "oracle_eval_F": (ctypes.c_int, [P, ctypes.c_double, dp, dp, dp]),
        "oracle_apply_J": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_double, dp, dp, dp]),
        "oracle_dense_J": (ctypes.c_int, [P, ctypes.c_double, dp, dp, lp]),
        "oracle_smooth": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_double, dp, dp, dp, ctypes.c_int]),
        "oracle_restrict": (ctypes.c_int, [P, ctypes.c_int, dp, dp]),
        "oracle_prolong": (ctypes.c_int, [P, ctypes.c_int, dp, dp]),
        "oracle_inject": (ctypes.c_int, [P, dp, ctypes.c_int, dp]),
        "oracle_cycles": (ctypes.c_int, [P, ctypes.c_double, dp, dp, dp, ctypes.c_int, dp]),
        "oracle_coarsest_matrix": (ctypes.c_int, [P, ctypes.c_double, dp, dp]),
        "oracle_coarsest_solve": (ctypes.c_int, [P, ctypes.c_double, dp, dp, dp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _l(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _b(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_byte))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class OracleError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"oracle error {code}: {msg}")
        self.code = code


class Oracle:
    """One domain: level-set geometry on [lo,hi]^dim with N intervals per axis.

    The state is the interleaved (s, c) of the finest level.  ``phi`` is given in
    (z,)y,x order with x fastest, shape (N+1,)*dim."""

    def __init__(self, phi, dim, lo, hi, N, coarsest_N=8):
        lib = _load()
        self.lib = lib
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        assert phi.size == (N + 1) ** dim
        st = ctypes.c_int(0)
        self.h = lib.oracle_create(_d(phi), dim, lo, hi, N, coarsest_N, ctypes.byref(st))
        if not self.h:
            raise OracleError(st.value, lib.oracle_last_error().decode())
        self.dim, self.N, self.lo, self.hi = dim, N, lo, hi
        self.shape = (N + 1,) * dim
        self.nn = (N + 1) ** dim
        self.nlev = lib.oracle_num_levels(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.oracle_destroy(self.h)
            self.h = None

    def _chk(self, rc):
        if rc != OK:
            raise OracleError(rc, self.lib.oracle_last_error().decode())

    def set_model(self, params):
        p = np.asarray(params, dtype=np.float64)
        self._chk(self.lib.oracle_set_model(self.h, _d(p)))

    def set_solver(self, nu1=2, nu2=2, cycle=1, max_newton=20, max_cycles=30, newton_tol=1e-10,
                   lin_rtol=1e-10, tau_s=0.9, smoother=0, ghost_sweeps=4):
        self._chk(self.lib.oracle_set_solver(self.h, nu1, nu2, cycle, max_newton, max_cycles, newton_tol,
                                             lin_rtol, tau_s, smoother, ghost_sweeps))

    def step(self, dt, nsteps=1):
        self._chk(self.lib.oracle_step(self.h, dt, nsteps))

    def get_state(self):
        s = np.zeros(self.nn)
        c = np.zeros(self.nn)
        t = np.zeros(self.nn, dtype=np.int8)
        self.lib.oracle_get_state(self.h, _d(s), _d(c), _b(t))
        return s.reshape(self.shape), c.reshape(self.shape), t.reshape(self.shape)

    def set_state(self, s, c, t=0.0):
        s = np.ascontiguousarray(s, dtype=np.float64).ravel()
        c = np.ascontiguousarray(c, dtype=np.float64).ravel()
        self._chk(self.lib.oracle_set_state(self.h, _d(s), _d(c), t))

    def stats(self):
        ist = np.zeros(5, dtype=np.int64)
        dst = np.zeros(3)
        self.lib.oracle_get_stats(self.h, _l(ist), _d(dst))
        return dict(newton_last=int(ist[0]), cycles_last=int(ist[1]), newton_total=int(ist[2]),
                    cycles_total=int(ist[3]), nrho=int(ist[4]), t=float(dst[0]), last_rho=float(dst[1]),
                    last_fnorm=float(dst[2]))

    def rho_history(self):
        n = self.stats()["nrho"]
        r = np.zeros(max(n, 1))
        f = np.zeros(max(n, 1), dtype=np.int8)
        n = self.lib.oracle_get_rho(self.h, _d(r), _b(f), n)
        return r[:n], f[:n].astype(bool)

    def clear_rho(self):
        self.lib.oracle_clear_rho(self.h)

    # ---- per-level inspection ----
    def level_info(self, l):
        info = np.zeros(8, dtype=np.int64)
        self._chk(self.lib.oracle_level_info(self.h, l, _l(info)))
        return dict(N=int(info[0]), n=int(info[1]), ng=int(info[2]), nb=int(info[3]), nact=int(info[4]),
                    kinds=(int(info[5]), int(info[6]), int(info[7])))

    def level_type(self, l):
        n = self.level_info(l)["n"]
        t = np.zeros(n ** self.dim, dtype=np.int8)
        self._chk(self.lib.oracle_level_type(self.h, l, _b(t)))
        return t

    def level_phi(self, l):
        n = self.level_info(l)["n"]
        p = np.zeros(n ** self.dim)
        self._chk(self.lib.oracle_level_phi(self.h, l, _d(p)))
        return p

    def level_ghosts(self, l):
        ng = self.level_info(l)["ng"]
        d = self.dim
        idx = np.zeros(max(ng, 1), dtype=np.int64)
        kind = np.zeros(max(ng, 1), dtype=np.int8)
        m = np.zeros(max(ng, 1) * d, dtype=np.int8)
        w = np.zeros(max(ng, 1) * d * 3)
        B = np.zeros(max(ng, 1) * d)
        self._chk(self.lib.oracle_level_ghosts(self.h, l, _l(idx), _b(kind), _b(m), _d(w), _d(B)))
        return dict(idx=idx[:ng], kind=kind[:ng], m=m[:ng * d].reshape(ng, d), w=w[:ng * d * 3].reshape(ng, d, 3),
                    B=B[:ng * d].reshape(ng, d))

    def level_rows(self, l):
        """Member weights of every ghost row (ng x 3^dim) and the unit normal of
        phi~ at each boundary point (ng x dim)."""
        ng = self.level_info(l)["ng"]
        d = self.dim
        K = 9 if d == 2 else 27
        wk = np.zeros(max(ng, 1) * K)
        nt = np.zeros(max(ng, 1) * d)
        self._chk(self.lib.oracle_level_rows(self.h, l, _d(wk), _d(nt)))
        return wk[:ng * K].reshape(ng, K), nt[:ng * d].reshape(ng, d)

    def set_bc(self, bc):
        """0: Dirichlet s = s_b (Eq. BCs); 1: Neumann ds/dn = s_b (Eq. BCsN)."""
        self._chk(self.lib.oracle_set_bc(self.h, int(bc)))

    def level_band(self, l):
        nb = self.level_info(l)["nb"]
        d = self.dim
        idx = np.zeros(max(nb, 1), dtype=np.int64)
        up = np.zeros(max(nb, 1) * d, dtype=np.int64)
        an = np.zeros(max(nb, 1) * d)
        self._chk(self.lib.oracle_level_band(self.h, l, _l(idx), _l(up), _d(an)))
        return dict(idx=idx[:nb], up=up[:nb * d].reshape(nb, d), an=an[:nb * d].reshape(nb, d))

    # ---- manufactured-solution inputs ----
    def set_ghost_sb(self, sb):
        if sb is None:
            self.lib.oracle_set_ghost_sb(self.h, None)
            return
        sb = np.ascontiguousarray(sb, dtype=np.float64)
        self._chk(self.lib.oracle_set_ghost_sb(self.h, _d(sb)))

    def set_sources(self, f1o=None, f1n=None, f2o=None, f2n=None):
        if f1o is None:
            self.lib.oracle_set_sources(self.h, None, None, None, None)
            return
        arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (f1o, f1n, f2o, f2n)]
        self._keep = arrs
        self._chk(self.lib.oracle_set_sources(self.h, *[_d(a) for a in arrs]))

    # ---- kernels of the method on explicit inputs (interleaved (s,c)) ----
    def eval_F(self, dt, W, Wn):
        W = np.ascontiguousarray(W, dtype=np.float64)
        Wn = np.ascontiguousarray(Wn, dtype=np.float64)
        F = np.zeros(2 * self.nn)
        self._chk(self.lib.oracle_eval_F(self.h, dt, _d(W), _d(Wn), _d(F)))
        return F

    def apply_J(self, l, dt, Wc, x):
        Wc = np.ascontiguousarray(Wc, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        self._chk(self.lib.oracle_apply_J(self.h, l, dt, _d(Wc), _d(x), _d(out)))
        return out

    def dense_J(self, dt, Wc):
        t = self.level_type(0)
        na = int(np.count_nonzero((t == 1) | (t == 2)))
        A = np.zeros((2 * na, 2 * na))
        act = np.zeros(na, dtype=np.int64)
        Wc = np.ascontiguousarray(Wc, dtype=np.float64)
        self.lib.oracle_dense_J(self.h, dt, _d(Wc), _d(A), _l(act))
        return A, act

    def smooth(self, l, dt, Wc, rhs, x, sweeps=1):
        x = np.array(x, dtype=np.float64)
        Wc = np.ascontiguousarray(Wc, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        self._chk(self.lib.oracle_smooth(self.h, l, dt, _d(Wc), _d(rhs), _d(x), sweeps))
        return x

    def restrict(self, l, res):
        res = np.array(res, dtype=np.float64)
        nc = self.level_info(l + 1)["n"] ** self.dim
        out = np.zeros(2 * nc)
        self._chk(self.lib.oracle_restrict(self.h, l, _d(res), _d(out)))
        return out, res

    def prolong(self, l, xc, xf):
        xc = np.ascontiguousarray(xc, dtype=np.float64)
        xf = np.array(xf, dtype=np.float64)
        self._chk(self.lib.oracle_prolong(self.h, l, _d(xc), _d(xf)))
        return xf

    def inject(self, Wc0, l):
        Wc0 = np.ascontiguousarray(Wc0, dtype=np.float64)
        out = np.zeros(2 * self.level_info(l)["n"] ** self.dim)
        self._chk(self.lib.oracle_inject(self.h, _d(Wc0), l, _d(out)))
        return out

    def coarsest_matrix(self, dt, Wc0):
        nact = self.level_info(self.nlev - 1)["nact"]
        A = np.zeros((2 * nact, 2 * nact))
        Wc0 = np.ascontiguousarray(Wc0, dtype=np.float64)
        self.lib.oracle_coarsest_matrix(self.h, dt, _d(Wc0), _d(A))
        return A

    def coarsest_solve(self, dt, Wc0, rhs_c):
        Wc0 = np.ascontiguousarray(Wc0, dtype=np.float64)
        rhs_c = np.ascontiguousarray(rhs_c, dtype=np.float64)
        x = np.zeros_like(rhs_c)
        self._chk(self.lib.oracle_coarsest_solve(self.h, dt, _d(Wc0), _d(rhs_c), _d(x)))
        return x

    def cycles(self, dt, Wc0, rhs, x, ncycles):
        Wc0 = np.ascontiguousarray(Wc0, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.array(x, dtype=np.float64)
        rn = np.zeros(ncycles)
        self._chk(self.lib.oracle_cycles(self.h, dt, _d(Wc0), _d(rhs), _d(x), ncycles, _d(rn)))
        return x, rn


def interleave(s, c):
    W = np.empty(2 * s.size)
    W[0::2] = np.ravel(s)
    W[1::2] = np.ravel(c)
    return W


def reinit(phi, dim, N, h, steps):
    """Reinitialization toward the signed distance (Sec. 2), oracle version."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    out = np.zeros_like(phi)
    rc = lib.oracle_reinit(_d(phi), dim, N, h, steps, _d(out))
    if rc:
        raise RuntimeError(f"oracle_reinit error {rc}")
    return out


def mask_levelset(mask, dim, N, steps):
    """Provisional level set of a binary mask (Sec. 2), oracle version."""
    lib = _load()
    m = np.ascontiguousarray(mask, dtype=np.int8)
    out = np.zeros(m.shape, dtype=np.float64)
    rc = lib.oracle_mask_levelset(m.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)), dim, N, steps, _d(out))
    if rc:
        raise RuntimeError(f"oracle_mask_levelset error {rc}")
    return out


def extrapolate(phi, types, u, dim, N, h, iters):
    """Linear extrapolation of u from the inside nodes to the rest of the box
    (the PDE approach used for the initial data, Sec. 3.3), oracle version."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    t = np.ascontiguousarray(types, dtype=np.int8)
    out = np.ascontiguousarray(u, dtype=np.float64).copy()
    rc = lib.oracle_extrapolate(_d(phi), t.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)), dim, N, h, iters, _d(out))
    if rc:
        raise RuntimeError(f"oracle_extrapolate error {rc}")
    return out
