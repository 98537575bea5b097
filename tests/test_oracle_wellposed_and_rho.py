"""Oracle pins of two measured facts (no GPU).

1. The 65^2 disk at dt = h has no discrete solution at its second CN step.
   The reaction rate k = (a/m_c) c0 ~ 999 gives k dt ~ 31 at h = 1/32.  The
   first step then extrapolates the ghosts to s ~ 9 and drives the ghost
   calcite negative.  At the second step the ghost c-equation of Eq. FDc,
   c/dt + (1/2)(a/m_s)(alpha c + beta) s c = c^n/dt - (1/2)(a/m_s) phi(c^n) s^n c^n,
   is a quadratic in c at given s_g.  It has no real root at some ghosts, so
   Newton cannot converge.  A quarter of the step (dt = h/4) is well posed and
   is what the small disk runs use.

2. Multigrid efficiency (Sec. 4.2): the convergence factor per cycle stays
   bounded as h -> 0.  On the paper's Test 3 geometry (disk R = 1.486,
   s0 = 0, c0 = 10, s_B = 1, dt = h, t in [0, 1]) with W(2,1) cycles the
   factors after the first few linear systems lie near 0.119 (Fig. rhohist).
"""
import numpy as np
import pytest

import workloads

PARAMS = workloads.PAPER_MODEL


def _ghost_c_discriminant(dt, s, s_old, c_old):
    """discriminant of A c^2 + B c + C = 0, the ghost c-equation of Eq. FDc at
    fixed s (CN average of the reaction term)"""
    a, d, m_s, m_c, alpha, beta = PARAMS[:6]
    k = a / m_s
    A = 0.5 * k * alpha * s
    B = 1.0 / dt + 0.5 * k * beta * s
    C = -c_old / dt + 0.5 * k * (alpha * c_old + beta) * s_old * c_old
    return B * B - 4.0 * A * C


def test_disk65_at_dt_h_has_no_discrete_solution(oracle_mod):
    N = 64
    dt = 2.0 / N
    o = oracle_mod.Oracle(workloads.disk(N), 2, -1.0, 1.0, N)
    o.set_model(PARAMS)
    o.set_solver()
    o.step(dt, 1)  # the first step converges
    s1, c1, t = o.get_state()
    g = t == 2
    assert c1[g].min() < 0.0 and s1[g].max() > 5.0  # the mechanism: overshooting ghosts
    with pytest.raises(oracle_mod.OracleError) as e:
        o.step(dt, 1)
    assert e.value.code == oracle_mod.ENOTCONV
    s2, _, _ = o.get_state()
    disc = _ghost_c_discriminant(dt, s2[g], s1[g], c1[g])
    assert np.sum(disc < 0.0) >= 1  # no real c at those ghosts for the iterate's s
    # the same disk with dt = h/4 runs the ten steps of the workload
    o2 = oracle_mod.Oracle(workloads.disk(N), 2, -1.0, 1.0, N)
    o2.set_model(PARAMS)
    o2.set_solver()
    o2.step(dt / 4, 10)
    s, c, t = o2.get_state()
    act = (t == 1) | (t == 2)
    assert np.all(np.isfinite(s[act])) and np.all(np.isfinite(c[act]))
    assert np.all(_ghost_c_discriminant(dt / 4, s[t == 2], s[t == 2], c[t == 2]) > 0)


def _rho_random_rhs(oracle_mod, o, dt, ncyc=12, seed=7):
    """geometric mean of the defect ratios of cycles 4..ncyc of a linear solve
    with the Jacobian at the current state and a seeded random right-hand side"""
    s, c, t = o.get_state()
    W = oracle_mod.interleave(s, c)
    act = ((t == 1) | (t == 2)).ravel()
    rng = np.random.default_rng(seed)
    rhs = np.zeros_like(W)
    rhs[0::2][act] = rng.standard_normal(act.sum())
    rhs[1::2][act] = rng.standard_normal(act.sum())
    _, rn = o.cycles(dt, W, rhs, np.zeros_like(W), ncyc)
    r = rn[3:] / rn[2:-1]
    return float(np.exp(np.mean(np.log(r))))


def test_convergence_factor_bounded_as_h_decreases(oracle_mod):
    """V(2,2) collective red-black cycles, Jacobian after one CN step at
    dt = h, star and disk, N = 64 ... 512: every factor is at most 0.3, none
    grows by more than 0.02 from one N to the next finer one past N = 128, and
    on the star (the benchmark geometry) the factors of N = 128 ... 512 lie
    within 0.05 of each other.  (The 4-level hierarchy of N = 64 converges
    more slowly: 0.21-0.26.)"""
    table = {}
    for geom in ("star", "disk"):
        for N in (64, 128, 256, 512):
            phi = workloads.star(N) if geom == "star" else workloads.disk(N)
            o = oracle_mod.Oracle(phi, 2, -1.0, 1.0, N)
            o.set_model(PARAMS)
            o.set_solver()
            o.step(2.0 / N, 1)
            table[geom, N] = _rho_random_rhs(oracle_mod, o, 2.0 / N)
    assert max(table.values()) <= 0.3, table
    for geom in ("star", "disk"):
        for N in (256, 512):
            assert table[geom, N] <= table[geom, N // 2] + 0.02, table
    star = [table["star", N] for N in (128, 256, 512)]
    assert max(star) - min(star) <= 0.05, table


@pytest.mark.parametrize("smoother", [2, 0], ids=["lexicographic", "red_black"])
def test_w21_convergence_factor_on_test3_geometry(oracle_mod, smoother):
    """Sec. 4.2, Test 3: W(2,1) cycles with collective Gauss-Seidel
    (lexicographic as in the paper, and red-black), N = 256 on [-2,2]^2 (the
    box is not given; R15), dt = h, t in [0, 1].  After the first five linear
    systems the median factor lies within 0.05 of the paper's 0.119."""
    N = 256
    h = 4.0 / N
    o = oracle_mod.Oracle(workloads.paper_test1(N), 2, -2.0, 2.0, N)
    o.set_model(PARAMS)
    o.set_solver(nu1=2, nu2=1, cycle=2, smoother=smoother)
    o.step(h, int(round(1.0 / h)))
    rho, first = o.rho_history()
    starts = np.nonzero(first)[0]
    assert len(starts) > 20
    late = rho[starts[5]:]
    late = late[~first[starts[5]:].astype(bool)]
    assert abs(np.median(late) - 0.119) <= 0.05, np.median(late)
