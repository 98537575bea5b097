"""More pins of the CPU oracle, aimed at its 3-D branch and at the star domain
(no GPU).

* Closed form of the residual: for s quadratic and c linear in the
  coordinates, the flux sum of L^s_h (Sec. 3.3, with the 1/h^2 of R1) equals
  d div(phi grad s) exactly, the tensor-quadratic boundary row (Eq. JssD)
  reproduces s at B, and F (Eqs. FDs, FDc, BCs) is known in closed form at
  every active node.  Distinct coefficients per axis make a wrong stride or a
  dropped neighbour on any axis show.
* Second order on manufactured solutions (Sec. 4.1) on the rounded box in 3-D
  and on the five-lobed star in 2-D.
* The heat-equation limit (a = 0) in 3-D.
"""
import numpy as np
import pytest

import workloads

PARAMS = workloads.PAPER_MODEL


def _poly_state(dim, N, lo, hi, Q, B, C0, gam, c0):
    """s = sum_{a<=b} Q[a][b] x_a x_b + sum_a B[a] x_a + C0 and
    c = c0 + sum_a gam[a] x_a at the nodes, with their exact derivatives."""
    X = workloads.node_coords(dim, lo, hi, N)
    s = C0 + sum(B[a] * X[a] for a in range(dim))
    for a in range(dim):
        for b in range(a, dim):
            s = s + Q[a][b] * X[a] * X[b]
    c = c0 + sum(gam[a] * X[a] for a in range(dim))
    grad = []
    for a in range(dim):
        g = B[a] + 2.0 * Q[a][a] * X[a]
        for b in range(dim):
            if b != a:
                g = g + Q[min(a, b)][max(a, b)] * X[b]
        grad.append(g)
    lap = 2.0 * sum(Q[a][a] for a in range(dim))
    return X, s, c, grad, lap


def _poly_value(dim, P, Q, B, C0):
    v = C0 + sum(B[a] * P[:, a] for a in range(dim))
    for a in range(dim):
        for b in range(a, dim):
            v = v + Q[a][b] * P[:, a] * P[:, b]
    return v


def _Ls_exact(P, s, c, grad, lap, gam):
    """L^s(s, c) = -(a/m_c) phi s c + d div(phi grad s) with phi = alpha c + beta"""
    a, d, m_s, m_c, alpha, beta = P[:6]
    ph = alpha * c + beta
    dot = sum(alpha * gam[k] * grad[k] for k in range(len(grad)))
    return -(a / m_c) * ph * s * c + d * (ph * lap + dot)


# the paper's constants, and the same without reaction (a = 0) so that the
# diffusion part, which the reaction term outweighs ~10^4 : 1, carries F^s alone
MODELS = {"paper": PARAMS, "no_reaction": (0.0,) + tuple(PARAMS[1:])}


@pytest.mark.parametrize("model", sorted(MODELS))
@pytest.mark.parametrize("dim,N,geom", [(2, 32, "star"), (3, 16, "rbox"), (3, 32, "rbox")])
def test_residual_closed_form_on_polynomial_states(oracle_mod, dim, N, geom, model):
    P = MODELS[model]
    phi = workloads.star(N, 0.6, 0.1) if geom == "star" else workloads.rounded_box(N)
    o = oracle_mod.Oracle(phi, dim, -1.0, 1.0, N, 4 if dim == 3 else 8)
    o.set_model(P)
    o.set_solver()
    a, d, m_s, m_c, alpha, beta = P[:6]
    s_ext = P[6]
    # iterate W and old state W^n, different polynomials, distinct per axis
    Q1 = [[0.7, 0.3, -0.2], [0.0, -1.3, 0.45], [0.0, 0.0, 2.1]]
    B1 = [0.25, -0.6, 0.9]
    Q0 = [[-0.4, 0.15, 0.35], [0.0, 0.8, -0.25], [0.0, 0.0, -1.7]]
    B0 = [-0.3, 0.5, 0.2]
    g1, g0 = [0.8, -1.9, 2.7], [-1.1, 0.6, 1.4]
    X, s1, c1, grad1, lap1 = _poly_state(dim, N, -1.0, 1.0, Q1, B1, 1.5, g1, 7.0)
    _, s0, c0, grad0, lap0 = _poly_state(dim, N, -1.0, 1.0, Q0, B0, 0.8, g0, 9.0)
    dt = 0.037
    W = oracle_mod.interleave(s1.ravel(), c1.ravel())
    Wn = oracle_mod.interleave(s0.ravel(), c0.ravel())
    F = o.eval_F(dt, W, Wn)
    t = o.level_type(0).reshape(s1.shape)
    ins, gh = t == 1, t == 2
    Fs, Fc = F[0::2].reshape(s1.shape), F[1::2].reshape(s1.shape)
    ph1, ph0 = alpha * c1 + beta, alpha * c0 + beta
    Fs_exact = (ph1 * s1 - ph0 * s0) / dt - 0.5 * (_Ls_exact(P, s0, c0, grad0, lap0, g0) +
                                                    _Ls_exact(P, s1, c1, grad1, lap1, g1))
    Fc_exact = (c1 - c0) / dt + 0.5 * (a / m_s) * (ph0 * s0 * c0 + ph1 * s1 * c1)
    Fs_in, Fs_in_exact = Fs[ins], Fs_exact[ins]
    if a == 0.0:  # the time term as well: F^s is then the diffusion part alone
        Fs_in = Fs_in - ((ph1 * s1 - ph0 * s0) / dt)[ins]
        Fs_in_exact = -0.5 * (_Ls_exact(P, s0, c0, grad0, lap0, g0) + _Ls_exact(P, s1, c1, grad1, lap1, g1))[ins]
    scale = np.abs(Fs_in_exact).max()
    assert np.abs(Fs_in - Fs_in_exact).max() <= 1e-11 * scale
    act = ins | gh
    assert np.abs(Fc[act] - Fc_exact[act]).max() <= 1e-12 * max(np.abs(Fc_exact[act]).max(), 1.0 / dt)
    # ghost rows: s~(B_g) - s_b, and s~ reproduces the quadratic at B
    g = o.level_ghosts(0)
    quad = g["kind"] == 0
    assert quad.sum() > 0.9 * len(quad)
    sB = _poly_value(dim, g["B"], Q1, B1, 1.5)
    flat = Fs.ravel()[g["idx"]]
    assert np.abs(flat[quad] - (sB[quad] - s_ext)).max() <= 1e-11 * np.abs(sB).max()


def _orders(errs):
    e = np.array(errs)
    return np.log2(e[:-1] / e[1:])


def test_manufactured_sources_3d_match_symbolic_derivation():
    pytest.importorskip("sympy")
    import manufactured as M

    rng = np.random.default_rng(8)
    X, Y, Z = (rng.uniform(-1, 1, 150) for _ in range(3))
    fs, fc, f1s, f2s = M.symbolic3(tuple(PARAMS[:6]))
    for t in (0.0, 0.29, 0.5):
        s, c = M.exact3(PARAMS[:6], X, Y, Z, t)
        f1, f2 = M.sources3(PARAMS[:6], X, Y, Z, t)
        assert np.allclose(s, fs(X, Y, Z, t), rtol=1e-14, atol=0)
        assert np.allclose(c, fc(X, Y, Z, t), rtol=1e-14, atol=0)
        assert np.allclose(f1, f1s(X, Y, Z, t), rtol=1e-12, atol=1e-9)
        assert np.allclose(f2, f2s(X, Y, Z, t), rtol=1e-12, atol=1e-9)


def test_second_order_on_manufactured_solution_3d_rounded_box(oracle_mod):
    """The manufactured-solution check of Sec. 4.1 carried to 3-D (the
    dimension-by-dimension extension): rounded box on [-1,1]^3, N = 16, 32, 64,
    dt = h, t = 0.25.  Errors of s and c fall at second order."""
    import manufactured as M

    errs = {}
    for N in (16, 32, 64):
        s, c, ty, XYZ, T = M.run_oracle3(oracle_mod, workloads.rounded_box(N), N, -1.0, 1.0, PARAMS[:6], 0.25)
        for k, v in M.rel_errors3(PARAMS[:6], s, c, ty, XYZ, T).items():
            errs.setdefault(k, []).append(v)
    for key in ("s_inf", "s_1", "c_inf", "c_1"):
        o = _orders(errs[key])
        assert o.mean() >= 1.8 and o.min() >= 1.6, (key, errs[key], o)


def test_second_order_on_manufactured_solution_star(oracle_mod):
    """Sec. 4.1's manufactured solution on the five-lobed star
    r - 0.6 - 0.2 sin 5 theta on [-1,1]^2, N = 64, 128, 256, dt = h, t = 0.25.
    The L1 errors of s, c and of their gradients fall at second order.  The
    max-norm errors converge too, but irregularly: at N = 128 and 256 they sit
    next to the few ghosts near the inward cusps whose rows fall back to linear
    interpolation (R6; 4 of 330 and 2 of 660 ghosts), so only their overall
    rate is bounded."""
    import manufactured as M

    errs = {}
    for N in (64, 128, 256):
        s, c, ty, X, Y, T = M.run_oracle(oracle_mod, workloads.star(N), N, -1.0, 1.0, PARAMS[:6], T=0.25)
        for k, v in M.rel_errors(PARAMS[:6], s, c, ty, X, Y, T, 2.0 / N).items():
            errs.setdefault(k, []).append(v)
    for key in ("s_1", "c_1", "gs_1", "gc_1"):
        o = _orders(errs[key])
        assert o.mean() >= 1.8 and o.min() >= 1.6, (key, errs[key], o)
    for key in ("s_inf", "c_inf"):
        assert np.log2(errs[key][0] / errs[key][-1]) / 2 >= 1.1, (key, errs[key])
        assert errs[key][-1] < 1e-6, (key, errs[key])


def test_heat_equation_limit_without_reaction_3d(oracle_mod):
    """a = 0 in 3-D: c stays c0 exactly, s -> s_ext (Eq. maineq); the slowest
    mode of the rounded box (half-width 0.8) decays like exp(-d pi^2 3/1.6^2 t)."""
    N = 16
    o = oracle_mod.Oracle(workloads.rounded_box(N), 3, -1.0, 1.0, N, 4)
    o.set_model((0.0,) + tuple(PARAMS[1:]))
    o.set_solver()
    o.step(0.1, 300)
    s, c, t = o.get_state()
    act = (t == 1) | (t == 2)
    assert np.abs(s[t == 1] - PARAMS[6]).max() < 1e-8
    assert np.all(c[act] == PARAMS[8])
