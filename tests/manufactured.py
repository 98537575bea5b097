"""Manufactured solution of the accuracy tests (Sec. 4.1): exact s, c and the
source terms f1, f2 that make them solve the sulfation system (Eq. maineq with
phi(c) = alpha c + beta).  The sources are written out by hand below; the CPU
test suite checks them against a symbolic derivation (sympy, where installed),
so this module itself needs only numpy."""
import numpy as np

R2, R3 = np.sqrt(2.0), np.sqrt(3.0)


def exact(params, X, Y, t):
    """s = 2 + sin x cos y sin(t + sqrt 2), c = 3 + sin(x/2) cos 3y sin(2t + sqrt 3)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    s = 2.0 + np.sin(X) * np.cos(Y) * np.sin(t + R2)
    c = 3.0 + np.sin(0.5 * X) * np.cos(3.0 * Y) * np.sin(2.0 * t + R3)
    return s, c


def sources(params, X, Y, t):
    """f1 = d/dt(phi s) + (a/m_c) phi s c - d div(phi grad s),
    f2 = dc/dt + (a/m_s) phi s c, by the product and chain rules."""
    a, d, m_s, m_c, alpha, beta = params
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    s, c = exact(params, X, Y, t)
    st, ct = np.sin(t + R2), np.sin(2.0 * t + R3)
    s_t = np.sin(X) * np.cos(Y) * np.cos(t + R2)
    c_t = 2.0 * np.sin(0.5 * X) * np.cos(3.0 * Y) * np.cos(2.0 * t + R3)
    s_x = np.cos(X) * np.cos(Y) * st
    s_y = -np.sin(X) * np.sin(Y) * st
    s_xx = -np.sin(X) * np.cos(Y) * st
    s_yy = -np.sin(X) * np.cos(Y) * st
    c_x = 0.5 * np.cos(0.5 * X) * np.cos(3.0 * Y) * ct
    c_y = -3.0 * np.sin(0.5 * X) * np.sin(3.0 * Y) * ct
    phi = alpha * c + beta
    div = alpha * c_x * s_x + phi * s_xx + alpha * c_y * s_y + phi * s_yy
    f1 = alpha * c_t * s + phi * s_t + (a / m_c) * phi * s * c - d * div
    f2 = c_t + (a / m_s) * phi * s * c
    return f1, f2


def exact_grad_s(params, X, Y, t):
    """Gradient of the exact s."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    st = np.sin(t + R2)
    return np.cos(X) * np.cos(Y) * st, -np.sin(X) * np.sin(Y) * st


def test_levelset(test, X, Y):
    """The level sets of Tests 1 and 2 (Sec. 4.1) as functions of the point."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if test.startswith("test1"):
        return np.sqrt((X - np.sqrt(2.0) / 30.0) ** 2 + (Y - np.sqrt(3.0) / 40.0) ** 2) - 1.486
    Lh, D = 0.9567, 0.3
    p1 = np.maximum(np.abs(X), np.abs(Y)) - Lh
    p2 = np.sqrt((np.abs(X) - Lh) ** 2 + (np.abs(Y) - Lh) ** 2) - D
    return np.minimum(p1, p2)


def boundary_normal(test, B):
    """Outward unit normal of the exact boundary at the points B (n x 2), from
    central differences of the level set function (step 1e-7)."""
    e = 1e-7
    gx = (test_levelset(test, B[:, 0] + e, B[:, 1]) - test_levelset(test, B[:, 0] - e, B[:, 1])) / (2 * e)
    gy = (test_levelset(test, B[:, 0], B[:, 1] + e) - test_levelset(test, B[:, 0], B[:, 1] - e)) / (2 * e)
    nrm = np.sqrt(gx * gx + gy * gy)
    return np.stack([gx / nrm, gy / nrm], 1)


def boundary_values(params, B, t, bc, normals=None):
    """s_b at the boundary points: s itself (Dirichlet), or (Neumann) the
    exact gradient of s along the given unit normals -- the discrete normals
    n~ of phi~ at B, as the scheme imposes them (Eq. BCsN): Test 2's boundary
    has corners where the exact normal jumps and no smooth normal exists."""
    if bc == 0:
        return exact(params, B[:, 0], B[:, 1], t)[0]
    sx, sy = exact_grad_s(params, B[:, 0], B[:, 1], t)
    return sx * normals[:, 0] + sy * normals[:, 1]


def symbolic(params):
    """The same exact solution and sources derived symbolically (sympy):
    (s, c, f1, f2) as numpy callables of (x, y, t)."""
    import sympy as sp

    a, d, m_s, m_c, alpha, beta = params
    x, y, t = sp.symbols("x y t", real=True)
    s = 2 + sp.sin(x) * sp.cos(y) * sp.sin(t + sp.sqrt(2))
    c = 3 + sp.sin(sp.Rational(1, 2) * x) * sp.cos(3 * y) * sp.sin(2 * t + sp.sqrt(3))
    phi = alpha * c + beta
    f1 = sp.diff(phi * s, t) + (a / m_c) * phi * s * c - d * (sp.diff(phi * sp.diff(s, x), x) +
                                                               sp.diff(phi * sp.diff(s, y), y))
    f2 = sp.diff(c, t) + (a / m_s) * phi * s * c
    mk = lambda e: sp.lambdify((x, y, t), e, "numpy")  # noqa: E731
    return mk(s), mk(c), mk(f1), mk(f2)


def run_oracle(oracle_mod, phi, N, lo, hi, params, T=1.0, dt_factor=1.0, bc=0):
    """Advance the oracle from the exact data at t = 0 to t = T with dt = h (the
    paper's choice, Sec. 4) and return (s, c, type, X, Y, T).  bc = 1 imposes
    the Neumann condition ds/dn = s_b of Sec. 3.6 with the exact normal
    derivative along the discrete normal as s_b."""
    import workloads

    X, Y = workloads.node_coords(2, lo, hi, N)
    h = (hi - lo) / N
    nsteps = int(round(T / (dt_factor * h)))
    dt = T / nsteps
    o = oracle_mod.Oracle(phi, 2, lo, hi, N)
    full = tuple(params) + (1.0, 0.0, 0.0)
    o.set_model(full)
    o.set_solver(newton_tol=1e-11)
    if bc:
        o.set_bc(bc)
    s0, c0 = exact(params, X, Y, 0.0)
    o.set_state(s0, c0, 0.0)
    g = o.level_ghosts(0)
    _, nt = o.level_rows(0)
    for k in range(nsteps):
        t0, t1 = k * dt, (k + 1) * dt
        f1o, f2o = sources(params, X, Y, t0)
        f1n, f2n = sources(params, X, Y, t1)
        o.set_sources(f1o, f1n, f2o, f2n)
        o.set_ghost_sb(boundary_values(params, g["B"], t1, bc, nt))
        o.step(dt, 1)
    s, c, ty = o.get_state()
    return s, c, ty, X, Y, nsteps * dt


def rel_errors(params, s, c, ty, X, Y, T, h):
    """Relative L1 and Linf errors of s and c on inside nodes, and of |grad s|,
    |grad c| by central differences on inside nodes whose four neighbours are
    active (Sec. 4.1)."""
    se, ce = exact(params, X, Y, T)
    ins = ty == 1
    out = {}
    for name, num, ex in (("s", s, se), ("c", c, ce)):
        e = np.abs(num - ex)[ins]
        out[name + "_inf"] = e.max() / np.abs(ex[ins]).max()
        out[name + "_1"] = e.sum() / np.abs(ex[ins]).sum()
        gx = (np.roll(num, -1, 1) - np.roll(num, 1, 1)) / (2 * h)
        gy = (np.roll(num, -1, 0) - np.roll(num, 1, 0)) / (2 * h)
        ex_gx = (np.roll(ex, -1, 1) - np.roll(ex, 1, 1)) / (2 * h)
        ex_gy = (np.roll(ex, -1, 0) - np.roll(ex, 1, 0)) / (2 * h)
        gn = np.sqrt(gx ** 2 + gy ** 2)
        ge = np.sqrt(ex_gx ** 2 + ex_gy ** 2)
        act = (ty == 1) | (ty == 2)
        ok = ins & np.roll(act, 1, 0) & np.roll(act, -1, 0) & np.roll(act, 1, 1) & np.roll(act, -1, 1)
        eg = np.abs(gn - ge)[ok]
        out["g" + name + "_inf"] = eg.max() / np.abs(ge[ok]).max()
        out["g" + name + "_1"] = eg.sum() / np.abs(ge[ok]).sum()
    return out


# ---- 3-D: the same construction on a rounded box (the dimension-by-dimension
# extension of the method; the paper's tests are 2-D) ----

def exact3(params, X, Y, Z, t):
    """s = 2 + sin x cos y cos z sin(t + sqrt 2),
    c = 3 + sin(x/2) cos 3y cos 2z sin(2t + sqrt 3)."""
    X, Y, Z = (np.asarray(A, dtype=np.float64) for A in (X, Y, Z))
    s = 2.0 + np.sin(X) * np.cos(Y) * np.cos(Z) * np.sin(t + R2)
    c = 3.0 + np.sin(0.5 * X) * np.cos(3.0 * Y) * np.cos(2.0 * Z) * np.sin(2.0 * t + R3)
    return s, c


def sources3(params, X, Y, Z, t):
    """f1 = d/dt(phi s) + (a/m_c) phi s c - d div(phi grad s),
    f2 = dc/dt + (a/m_s) phi s c, written out by hand in 3-D."""
    a, d, m_s, m_c, alpha, beta = params
    X, Y, Z = (np.asarray(A, dtype=np.float64) for A in (X, Y, Z))
    s, c = exact3(params, X, Y, Z, t)
    st, ct = np.sin(t + R2), np.sin(2.0 * t + R3)
    sx, cy, cz = np.sin(X), np.cos(Y), np.cos(Z)
    s_t = sx * cy * cz * np.cos(t + R2)
    s_x = np.cos(X) * cy * cz * st
    s_y = -sx * np.sin(Y) * cz * st
    s_z = -sx * cy * np.sin(Z) * st
    lap_s = -3.0 * sx * cy * cz * st
    hx, c3y, c2z = np.sin(0.5 * X), np.cos(3.0 * Y), np.cos(2.0 * Z)
    c_t = 2.0 * hx * c3y * c2z * np.cos(2.0 * t + R3)
    c_x = 0.5 * np.cos(0.5 * X) * c3y * c2z * ct
    c_y = -3.0 * hx * np.sin(3.0 * Y) * c2z * ct
    c_z = -2.0 * hx * c3y * np.sin(2.0 * Z) * ct
    phi = alpha * c + beta
    div = alpha * (c_x * s_x + c_y * s_y + c_z * s_z) + phi * lap_s
    f1 = alpha * c_t * s + phi * s_t + (a / m_c) * phi * s * c - d * div
    f2 = c_t + (a / m_s) * phi * s * c
    return f1, f2


def symbolic3(params):
    """exact3 and sources3 derived symbolically (sympy): numpy callables of
    (x, y, z, t)."""
    import sympy as sp

    a, d, m_s, m_c, alpha, beta = params
    x, y, z, t = sp.symbols("x y z t", real=True)
    s = 2 + sp.sin(x) * sp.cos(y) * sp.cos(z) * sp.sin(t + sp.sqrt(2))
    c = 3 + sp.sin(x / 2) * sp.cos(3 * y) * sp.cos(2 * z) * sp.sin(2 * t + sp.sqrt(3))
    phi = alpha * c + beta
    div = sum(sp.diff(phi * sp.diff(s, v), v) for v in (x, y, z))
    f1 = sp.diff(phi * s, t) + (a / m_c) * phi * s * c - d * div
    f2 = sp.diff(c, t) + (a / m_s) * phi * s * c
    mk = lambda e: sp.lambdify((x, y, z, t), e, "numpy")  # noqa: E731
    return mk(s), mk(c), mk(f1), mk(f2)


def run_oracle3(oracle_mod, phi, N, lo, hi, params, T, coarsest_N=4):
    """Advance the oracle in 3-D from the exact data at t = 0 to t = T with
    dt = h, Dirichlet data s_b = exact s at each ghost's boundary point B_g
    and t_{n+1}, CN-averaged sources.  Returns (s, c, type, (X, Y, Z), T)."""
    import workloads

    X, Y, Z = workloads.node_coords(3, lo, hi, N)
    h = (hi - lo) / N
    nsteps = max(1, int(round(T / h)))
    dt = T / nsteps
    o = oracle_mod.Oracle(phi, 3, lo, hi, N, coarsest_N)
    o.set_model(tuple(params) + (1.0, 0.0, 0.0))
    o.set_solver(newton_tol=1e-11)
    s0, c0 = exact3(params, X, Y, Z, 0.0)
    o.set_state(s0, c0, 0.0)
    B = o.level_ghosts(0)["B"]
    for k in range(nsteps):
        t0, t1 = k * dt, (k + 1) * dt
        f1o, f2o = sources3(params, X, Y, Z, t0)
        f1n, f2n = sources3(params, X, Y, Z, t1)
        o.set_sources(f1o, f1n, f2o, f2n)
        o.set_ghost_sb(exact3(params, B[:, 0], B[:, 1], B[:, 2], t1)[0])
        o.step(dt, 1)
    s, c, ty = o.get_state()
    return s, c, ty, (X, Y, Z), nsteps * dt


def rel_errors3(params, s, c, ty, XYZ, T):
    """Relative L1 and Linf errors of s and c on the inside nodes (3-D)."""
    se, ce = exact3(params, *XYZ, T)
    ins = ty == 1
    out = {}
    for name, num, ex in (("s", s, se), ("c", c, ce)):
        e = np.abs(num - ex)[ins]
        out[name + "_inf"] = e.max() / np.abs(ex[ins]).max()
        out[name + "_1"] = e.sum() / np.abs(ex[ins]).sum()
    return out
