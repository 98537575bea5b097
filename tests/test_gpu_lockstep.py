"""Lock-step batching: the instances of one size class advance their Newton
iterations and multigrid cycles together, each phase of a cycle (Sec. 3.5) one
launch over all of them.  Every instance must run the iterations and cycles it
runs alone and reach the CPU oracle's result within the whole-run tolerances
(1e-10 relative in max-norm over the active nodes for the FP64 form, 1e-8 for
mixed precision); against the same instance stepped alone the FP64 form agrees
to 1e-12 (only the rounding order of a few reductions differs)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

RUN_TOL = 1e-10
MIXED_TOL = 1e-8
ALONE_TOL = 1e-12


def _close(a, b, tol):
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max() / scale
    assert err <= tol, f"relative error {err:.3e} > {tol:.1e}"
    return err


def _star_spec(N, seed, cN=8):
    a, p, s_ext = workloads.random_star_params(np.random.default_rng(seed))
    model = list(workloads.PAPER_MODEL)
    model[6] = s_ext
    return dict(phi=workloads.random_star(N, a, p), dim=2, N=N, cN=cN, model=model, dt=2.0 / N, nsteps=2)


def _box_spec(N, s_ext):
    model = list(workloads.PAPER_MODEL)
    model[6] = s_ext
    return dict(phi=workloads.rounded_box(N), dim=3, N=N, cN=8, model=model, dt=0.25 * 2.0 / N, nsteps=1)


def _specs():
    # a 2-D class of four stars, a 3-D class of two boxes, and a star of its
    # own size (which runs alone)
    sp = [_star_spec(128, 700 + k) for k in range(4)]
    sp += [_box_spec(32, 1.0), _box_spec(32, 0.7)]
    sp.append(_star_spec(96, 710, cN=6))
    return sp


def _domain(sulfmg, sp, **solver):
    d = sulfmg.Domain(sp["phi"], sp["dim"], (-1.0, 1.0), sp["N"], sp["cN"])
    d.set_model(sp["model"])
    if sp.get("bc"):
        d.set_bc(sp["bc"])
    d.set_solver(**solver)
    return d


def _run_lockstep(sulfmg, specs, nstreams=2, **solver):
    doms = [_domain(sulfmg, sp, **solver) for sp in specs]
    batch = sulfmg.Batch(doms, nstreams=nstreams, lockstep=True)
    batch.step([sp["dt"] for sp in specs], [sp["nsteps"] for sp in specs])
    st = list(batch.status())
    batch.close()
    out = []
    for d in doms:
        out.append((d.get_state(), d.stats()))
        d.close()
    return st, out


@pytest.mark.parametrize("precision", [0, 1])
def test_lockstep_matches_oracle(sulfmg, oracle_mod, precision):
    specs = _specs()
    st, out = _run_lockstep(sulfmg, specs, precision=precision)
    assert st == [0] * len(specs)
    tol = RUN_TOL if precision == 0 else MIXED_TOL
    for sp, ((s, c, t), stats) in zip(specs, out):
        ref = oracle_mod.Oracle(sp["phi"], sp["dim"], -1.0, 1.0, sp["N"], sp["cN"])
        ref.set_model(sp["model"])
        ref.set_solver()
        ref.step(sp["dt"], sp["nsteps"])
        rs, rc, rt = ref.get_state()
        assert np.array_equal(t, rt)
        act = (rt == 1) | (rt == 2)
        _close(s[act], rs[act], tol)
        _close(c[act], rc[act], tol)
        assert stats["steps_total"] == sp["nsteps"]
        assert abs(stats["t"] - sp["dt"] * sp["nsteps"]) <= 1e-15


@pytest.mark.parametrize("precision,mf", [(0, 1), (1, 1), (1, 0)])
def test_lockstep_equals_alone(sulfmg, precision, mf):
    """same Newton iterations and cycles as alone, results to rounding (FP64
    1e-12; mixed precision, matrix-free or stored FP32 coefficients, 1e-8)"""
    specs = _specs()
    st, out = _run_lockstep(sulfmg, specs, nstreams=3, precision=precision, relax_matrix_free=mf)
    assert st == [0] * len(specs)
    tol = ALONE_TOL if precision == 0 else MIXED_TOL
    for sp, ((s, c, t), stats) in zip(specs, out):
        d = _domain(sulfmg, sp, precision=precision, relax_matrix_free=mf)
        d.step(sp["dt"], sp["nsteps"])
        s1, c1, _ = d.get_state()
        a = d.stats()
        d.close()
        act = (t == 1) | (t == 2)
        _close(s[act], s1[act], tol)
        _close(c[act], c1[act], tol)
        assert stats["newton_total"] == a["newton_total"]
        if precision == 0:
            assert stats["cycles_total"] == a["cycles_total"]
        else:
            assert abs(stats["cycles_total"] - a["cycles_total"]) <= sp["nsteps"]


def test_lockstep_one_stream_and_repeated_calls(sulfmg):
    """a class split over two step calls and run on one worker equals one call
    of two steps"""
    specs = [_star_spec(128, 720 + k) for k in range(3)]
    doms = [_domain(sulfmg, sp) for sp in specs]
    batch = sulfmg.Batch(doms, nstreams=1, lockstep=True)
    batch.step(2.0 / 128, 1)
    batch.step(2.0 / 128, 1)
    assert list(batch.status()) == [0, 0, 0]
    batch.close()
    _, out = _run_lockstep(sulfmg, specs)
    for d, ((s, c, t), _) in zip(doms, out):
        s1, c1, _ = d.get_state()
        assert d.stats()["steps_total"] == 2
        d.close()
        assert np.array_equal(s, s1) and np.array_equal(c, c1)


def test_lockstep_failing_instance_is_isolated(sulfmg):
    """two 65^2 disks at dt = h in one class: with the paper's reaction rate
    the CN system of the second step has no solution (Newton reports
    ENOTCONV), with a tenth of it every step converges; the failure leaves the
    other instance's steps untouched"""
    good = list(workloads.PAPER_MODEL)
    good[0] = 1.0e3
    specs = [dict(phi=workloads.disk(64), dim=2, N=64, cN=8, model=m, dt=2.0 / 64, nsteps=10)
             for m in (list(workloads.PAPER_MODEL), good)]
    doms = [_domain(sulfmg, sp) for sp in specs]
    batch = sulfmg.Batch(doms, nstreams=1, lockstep=True)
    with pytest.raises(sulfmg.SulfError) as e:
        batch.step(2.0 / 64, 10)
    assert e.value.code == sulfmg.ENOTCONV
    assert list(batch.status()) == [sulfmg.ENOTCONV, 0]
    batch.close()
    assert doms[0].stats()["steps_total"] < 10
    assert doms[1].stats()["steps_total"] == 10
    s, c, t = doms[1].get_state()
    d = _domain(sulfmg, specs[1])
    d.step(2.0 / 64, 10)
    s1, c1, _ = d.get_state()
    d.close()
    act = (t == 1) | (t == 2)
    _close(s[act], s1[act], ALONE_TOL)
    _close(c[act], c1[act], ALONE_TOL)
    for x in doms:
        x.close()


def test_ineligible_solver_runs_alone(sulfmg):
    """W-cycles cannot join a class: in lock-step mode such instances run
    alone, bit for bit as in the default mode"""
    specs = [_star_spec(128, 730 + k) for k in range(2)]
    res = []
    for lock in (False, True):
        doms = [_domain(sulfmg, sp, cycle=2, nu1=2, nu2=1) for sp in specs]
        batch = sulfmg.Batch(doms, nstreams=2, lockstep=lock)
        batch.step(2.0 / 128, 1)
        batch.close()
        res.append([d.get_state()[:2] for d in doms])
        for d in doms:
            d.close()
    for (s0, c0), (s1, c1) in zip(*res):
        assert np.array_equal(s0, s1) and np.array_equal(c0, c1)


@pytest.mark.parametrize("precision", [0, 1])
def test_lockstep_graphs_are_bitwise_neutral(sulfmg, precision):
    """the phases replayed from captured graphs (with the per-instance work on
    parallel branches) compute exactly what direct launches compute"""
    specs = [_star_spec(128, 740 + k) for k in range(5)] + [_box_spec(32, 0.9), _box_spec(32, 0.6)]
    runs = [_run_lockstep(sulfmg, specs, precision=precision, graphs=g) for g in (0, 1)]
    for (st0, o0), (st1, o1) in [runs]:
        assert st0 == st1 == [0] * len(specs)
        for ((s0, c0, _), a0), ((s1, c1, _), a1) in zip(o0, o1):
            assert np.array_equal(s0, s1) and np.array_equal(c0, c1)
            assert a0["cycles_total"] == a1["cycles_total"] and a0["newton_total"] == a1["newton_total"]


@pytest.mark.parametrize("precision", [0, 1])
def test_lockstep_neumann_coarsest4_without_dependent_launch(sulfmg, oracle_mod, precision):
    """a class of Neumann stars (Sec. 3.6 rows) and a class of 3-D boxes whose
    hierarchy ends at a 5^3 coarsest grid, stepped in lock step with dependent
    launch off, against the oracle"""
    sp = []
    for k in range(3):
        x = _star_spec(128, 750 + k)
        x.update(bc=1, dt=0.25 * 2.0 / 128)
        sp.append(x)
    for s_ext in (1.0, 0.8):
        x = _box_spec(32, s_ext)
        x.update(cN=4)
        sp.append(x)
    st, out = _run_lockstep(sulfmg, sp, precision=precision, pdl=0)
    assert st == [0] * len(sp)
    tol = RUN_TOL if precision == 0 else MIXED_TOL
    for x, ((s, c, t), stats) in zip(sp, out):
        ref = oracle_mod.Oracle(x["phi"], x["dim"], -1.0, 1.0, x["N"], x["cN"])
        ref.set_model(x["model"])
        if x.get("bc"):
            ref.set_bc(x["bc"])
        ref.set_solver()
        ref.step(x["dt"], x["nsteps"])
        rs, rc, rt = ref.get_state()
        act = (rt == 1) | (rt == 2)
        _close(s[act], rs[act], tol)
        _close(c[act], rc[act], tol)
        assert stats["steps_total"] == x["nsteps"]
