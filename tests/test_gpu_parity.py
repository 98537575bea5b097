"""GPU parity: every stage of the CUDA path against the CPU oracle on the same
seeded inputs, then whole Crank-Nicolson steps (arXiv:1902.07029, Sec. 3).

Tolerances: a single kernel application in FP64 agrees to 1e-12 relative to
the magnitude of the compared quantity (only the rounding order differs: FMA
contraction, summation order); whole runs to 1e-10 relative in max-norm over
the active nodes (FP64 form) and 1e-8 (mixed precision)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

STAGE_TOL = 1e-12
RUN_TOL = 1e-10
MIXED_TOL = 1e-8


def _pair(sulfmg, oracle_mod, phi, dim, N, coarsest=8, lo=-1.0, hi=1.0):
    dom = sulfmg.Domain(phi, dim, (lo, hi), N, coarsest)
    ref = oracle_mod.Oracle(phi, dim, lo, hi, N, coarsest)
    dom.set_model(workloads.PAPER_MODEL)
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    return dom, ref


def _rand_state(rng, t):
    act = (t == 1) | (t == 2)
    W = np.zeros(2 * t.size)
    W[0::2][act] = rng.uniform(0.0, 1.0, act.sum())
    W[1::2][act] = rng.uniform(5.0, 10.0, act.sum())
    return W


def _rand_vec(rng, t):
    act = (t == 1) | (t == 2)
    v = np.zeros(2 * t.size)
    v[0::2][act] = rng.standard_normal(act.sum())
    v[1::2][act] = rng.standard_normal(act.sum())
    return v


def _close(a, b, tol):
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max() / scale
    assert err <= tol, f"relative error {err:.3e} > {tol:.1e}"
    return err


GEOMS = [
    ("disk64", lambda: (workloads.disk(64), 2, 64, 8)),
    ("star256", lambda: (workloads.star(256), 2, 256, 8)),
    ("offdisk48", lambda: (workloads.disk(48, 0.55, (0.13, -0.07)), 2, 48, 6)),
    ("rbox32", lambda: (workloads.rounded_box(32), 3, 32, 8)),
]


@pytest.mark.parametrize("name,mk", GEOMS, ids=[g[0] for g in GEOMS])
def test_geometry(sulfmg, oracle_mod, name, mk):
    phi, dim, N, cN = mk()
    dom, ref = _pair(sulfmg, oracle_mod, phi, dim, N, cN)
    for l in range(ref.nlev):
        assert np.array_equal(dom.level_type(l), ref.level_type(l)), f"type differs at level {l}"
        gd, go = dom.level_ghosts(l), ref.level_ghosts(l)
        assert np.array_equal(gd["idx"], go["idx"])
        assert np.array_equal(gd["kind"], go["kind"])
        assert np.array_equal(gd["m"], go["m"])
        assert np.abs(gd["w"] - go["w"]).max() <= 1e-11
        assert np.abs(gd["B"] - go["B"]).max() <= 1e-12
        li, lo_ = dom.level_info(l), ref.level_info(l)
        assert (li["ng"], li["nb"], li["nact"]) == (lo_["ng"], lo_["nb"], lo_["nact"])


@pytest.mark.parametrize("name,mk", GEOMS, ids=[g[0] for g in GEOMS])
def test_stages(sulfmg, oracle_mod, name, mk):
    phi, dim, N, cN = mk()
    dom, ref = _pair(sulfmg, oracle_mod, phi, dim, N, cN)
    rng = np.random.default_rng(7)
    dt = 2.0 / N
    t0 = ref.level_type(0)
    W, Wn = _rand_state(rng, t0), _rand_state(rng, t0)
    _close(dom.eval_F(dt, W, Wn), ref.eval_F(dt, W, Wn), STAGE_TOL)
    for l in range(ref.nlev):
        tl = ref.level_type(l)
        Wc, x, rhs = _rand_state(rng, tl), _rand_vec(rng, tl), _rand_vec(rng, tl)
        _close(dom.apply_J(l, dt, Wc, x), ref.apply_J(l, dt, Wc, x), STAGE_TOL)
        # the ghost passes composed into one map per ghost (default) and pass by pass
        info = dom.level_info(l)
        if info["ng"] > 0:
            assert info["ghost_map_passes"] == 4 and 0 < info["ghost_map_entries"] <= 27 * info["ng"]
        for compose in (1, 0):
            dom.set_solver(ghost_compose=compose)
            _close(dom.smooth(l, dt, Wc, rhs, x, 1), ref.smooth(l, dt, Wc, rhs, x, 1), STAGE_TOL)
            _close(dom.smooth(l, dt, Wc, rhs, x, 3), ref.smooth(l, dt, Wc, rhs, x, 3), 1e-11)
        dom.set_solver()
        if l + 1 < ref.nlev:
            res = _rand_vec(rng, tl)
            cg, fg = dom.restrict(l, res)
            co, fo = ref.restrict(l, res)
            _close(fg, fo, STAGE_TOL)
            _close(cg, co, STAGE_TOL)
            xc = _rand_vec(rng, ref.level_type(l + 1))
            _close(dom.prolong(l, xc, x), ref.prolong(l, xc, x), STAGE_TOL)
    W0 = _rand_state(rng, t0)
    for l in range(1, ref.nlev):
        _close(dom.inject(W0, l), ref.inject(W0, l), STAGE_TOL)


@pytest.mark.parametrize("fuse_below", [100000, 0], ids=["fused_coarse", "per_level"])
@pytest.mark.parametrize("name,mk", GEOMS, ids=[g[0] for g in GEOMS])
def test_cycles(sulfmg, oracle_mod, name, mk, fuse_below):
    """cycles with the coarse levels fused into one single-CTA kernel and with
    every level as separate kernels"""
    phi, dim, N, cN = mk()
    dom, ref = _pair(sulfmg, oracle_mod, phi, dim, N, cN)
    dom.set_solver(fuse_below=fuse_below)
    rng = np.random.default_rng(11)
    dt = 2.0 / N
    t0 = ref.level_type(0)
    W = _rand_state(rng, t0)
    rhs = _rand_vec(rng, t0)
    xg, rg = dom.cycles(dt, W, rhs, 4)
    xo, ro = ref.cycles(dt, W, rhs, np.zeros_like(rhs), 4)
    _close(xg, xo, 1e-10)
    assert np.all(np.abs(rg - ro) <= 1e-10 * np.abs(ro))
    # the coarsest-level direct solve on its own
    tc = ref.level_type(ref.nlev - 1)
    bc = _rand_vec(rng, tc)
    _close(dom.coarsest_solve(dt, W, bc), ref.coarsest_solve(dt, W, bc), 1e-11)


RUNS = [
    ("disk64_dt_h/4", lambda: (workloads.disk(64), 2, 64, 8, 0.25 * 2.0 / 64, 10)),
    ("disk128", lambda: (workloads.disk(128), 2, 128, 8, 2.0 / 128, 5)),
    ("star256", lambda: (workloads.star(256), 2, 256, 8, 2.0 / 256, 3)),
    ("offdisk96_coarse6", lambda: (workloads.disk(96, 0.55, (0.13, -0.07)), 2, 96, 6, 0.25 * 2.0 / 96, 3)),
    ("rbox32_3d", lambda: (workloads.rounded_box(32), 3, 32, 8, 0.25 * 2.0 / 32, 2)),
]


@pytest.mark.parametrize("name,mk", RUNS, ids=[r[0] for r in RUNS])
def test_steps_fp64(sulfmg, oracle_mod, name, mk):
    phi, dim, N, cN, dt, nsteps = mk()
    dom, ref = _pair(sulfmg, oracle_mod, phi, dim, N, cN)
    dom.set_solver(fuse_below=4000)  # level 0 (and 1) as separate kernels, the coarser levels fused
    dom.step(dt, nsteps)
    ref.step(dt, nsteps)
    s, c, t = dom.get_state()
    rs, rc, rt = ref.get_state()
    assert np.array_equal(t, rt)
    act = (rt == 1) | (rt == 2)
    _close(s[act], rs[act], RUN_TOL)
    _close(c[act], rc[act], RUN_TOL)
    sd, so = dom.stats(), ref.stats()
    assert sd["steps_total"] == nsteps


@pytest.mark.parametrize("name,mk", RUNS[1:3], ids=[r[0] for r in RUNS[1:3]])
def test_steps_unfused_and_w_cycle(sulfmg, oracle_mod, name, mk):
    """every level as separate kernels without graphs, and the paper's W-cycle"""
    phi, dim, N, cN, dt, nsteps = mk()
    for kw in (dict(fuse_below=0, graphs=0), dict(cycle=2, nu1=2, nu2=1), dict(pdl=0), dict(ghost_compose=0),
               dict(ghost_sweeps=2, tau_s=0.7)):
        dom, ref = _pair(sulfmg, oracle_mod, phi, dim, N, cN)
        dom.set_solver(**kw)
        ref.set_solver(**{k: v for k, v in kw.items() if k in ("cycle", "nu1", "nu2", "ghost_sweeps", "tau_s")})
        dom.step(dt, nsteps)
        ref.step(dt, nsteps)
        s, c, t = dom.get_state()
        rs, rc, rt = ref.get_state()
        act = (rt == 1) | (rt == 2)
        _close(s[act], rs[act], RUN_TOL)
        _close(c[act], rc[act], RUN_TOL)


@pytest.mark.parametrize("precision", [0, 1])
def test_device_cycle_loop_is_bitwise_neutral(sulfmg, precision):
    """the cycles of a linear solve run as one graph launch (a conditional
    while node, convergence tested on the device) compute exactly what one
    launch and host test per cycle compute, with the same cycle counts"""
    phi, dim, N, cN, dt, nsteps = RUNS[2][1]()
    out, stats = [], []
    for prof in (0, 1):  # profiling events force the per-cycle host loop
        dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N, coarsest_N=cN)
        dom.set_model(workloads.PAPER_MODEL)
        dom.set_solver(precision=precision)
        dom.set_profiling(prof)
        dom.step(dt, nsteps)
        out.append(dom.get_state()[:2])
        stats.append(dom.stats())
        dom.close()
    assert stats[0]["loop_graph"] == 1 and stats[1]["loop_graph"] == 0
    assert stats[0]["cycles_total"] == stats[1]["cycles_total"]
    assert stats[0]["newton_total"] == stats[1]["newton_total"]
    assert abs(stats[0]["last_rho"] - stats[1]["last_rho"]) <= 1e-12
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("name,mk", RUNS[:3], ids=[r[0] for r in RUNS[:3]])
def test_steps_mixed(sulfmg, oracle_mod, name, mk):
    phi, dim, N, cN, dt, nsteps = mk()
    dom, ref = _pair(sulfmg, oracle_mod, phi, dim, N, cN)
    dom.set_solver(precision=1)
    dom.step(dt, nsteps)
    ref.step(dt, nsteps)
    s, c, t = dom.get_state()
    rs, rc, rt = ref.get_state()
    act = (rt == 1) | (rt == 2)
    _close(s[act], rs[act], MIXED_TOL)
    _close(c[act], rc[act], MIXED_TOL)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,mk", [RUNS[2], RUNS[4]], ids=[RUNS[2][0], RUNS[4][0]])
def test_dependent_launch_is_bitwise_neutral(sulfmg, name, mk, precision):
    """programmatic dependent launch only changes when a kernel is scheduled,
    never what it computes: the state after a few steps is bit for bit the
    same with it on and off, with and without graphs"""
    phi, dim, N, cN, dt, nsteps = mk()
    out = []
    for kw in (dict(pdl=1), dict(pdl=0), dict(pdl=1, graphs=0, fuse_below=0), dict(pdl=1, relax_occupancy=1)):
        dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N, coarsest_N=cN)
        dom.set_model(workloads.PAPER_MODEL)
        dom.set_solver(precision=precision, **kw)
        dom.step(dt, nsteps)
        out.append(dom.get_state()[:2])
        dom.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    # the higher-occupancy build of the FP64 relaxation computes the same bits
    assert np.array_equal(out[0][0], out[3][0]) and np.array_equal(out[0][1], out[3][1])
    # launched one by one, every level as separate kernels: same up to the
    # summation order of the coarsest solve
    for a, b in zip(out[0], out[2]):
        assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(b)), 1.0)


@pytest.mark.parametrize("name,mk", [RUNS[2], RUNS[4]], ids=[RUNS[2][0], RUNS[4][0]])
def test_matrix_free_fp32_relaxation(sulfmg, oracle_mod, name, mk):
    """the FP32 relaxation that recomputes its coefficients from (s, c) forms
    the stored coefficients' numbers: the mixed-precision steps agree with the
    stored-coefficient kernel and with the oracle (1e-8)"""
    phi, dim, N, cN, dt, nsteps = mk()
    out = []
    for mf in (0, 1):
        dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N, coarsest_N=cN)
        dom.set_model(workloads.PAPER_MODEL)
        dom.set_solver(precision=1, relax_matrix_free=mf)
        dom.step(dt, nsteps)
        out.append(dom.get_state())
        dom.close()
    ref = oracle_mod.Oracle(phi, dim, -1.0, 1.0, N, cN)
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    ref.step(dt, nsteps)
    rs, rc, rt = ref.get_state()
    act = (rt == 1) | (rt == 2)
    for s, c, _ in out:
        _close(s[act], rs[act], MIXED_TOL)
        _close(c[act], rc[act], MIXED_TOL)
    _close(out[1][0][act], out[0][0][act], 1e-12)
    _close(out[1][1][act], out[0][1][act], 1e-12)


def test_tiled_fp32_sweep(sulfmg, oracle_mod):
    """the temporally blocked FP32 sweep (both colours in one kernel, 3-D
    levels with >= 100k inside nodes) gives the two colour launches' numbers:
    the mixed-precision steps agree with the per-colour matrix-free kernel
    and with the oracle (1e-8)"""
    N, cN = 64, 4
    phi = workloads.rounded_box(N)
    dt = 0.25 * 2.0 / N
    out, cyc = [], []
    for mf in (1, 2):
        dom = sulfmg.Domain(phi, 3, (-1.0, 1.0), N, coarsest_N=cN)
        dom.set_model(workloads.PAPER_MODEL)
        dom.set_solver(precision=1, relax_matrix_free=mf)
        dom.step(dt, 2)
        out.append(dom.get_state())
        cyc.append(dom.stats()["cycles_total"])
        dom.close()
    ref = oracle_mod.Oracle(phi, 3, -1.0, 1.0, N, cN)
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    ref.step(dt, 2)
    rs, rc, rt = ref.get_state()
    act = (rt == 1) | (rt == 2)
    for s, c, _ in out:
        _close(s[act], rs[act], MIXED_TOL)
        _close(c[act], rc[act], MIXED_TOL)
    _close(out[1][0][act], out[0][0][act], 1e-12)
    _close(out[1][1][act], out[0][1][act], 1e-12)
    assert cyc[0] == cyc[1]
