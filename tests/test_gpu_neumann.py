"""The Neumann boundary condition for s (Sec. 3.6) on the GPU: boundary rows,
CN steps in FP64 and mixed precision against the oracle, and the accuracy
tests 1N/2N of Sec. 4.1 on the device."""
import json
import os

import numpy as np
import pytest

import manufactured as M
import workloads

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
RUN_TOL = 1e-10
MIXED_TOL = 1e-8


def _pair(sulfmg, oracle_mod, phi, dim, N, coarsest=8):
    dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N, coarsest)
    ref = oracle_mod.Oracle(phi, dim, -1.0, 1.0, N, coarsest)
    dom.set_model(workloads.PAPER_MODEL)
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    dom.set_bc(1)
    ref.set_bc(1)
    return dom, ref


def _close(a, b, tol):
    scale = max(np.max(np.abs(b)), 1e-300)
    assert np.max(np.abs(a - b)) <= tol * scale, np.max(np.abs(a - b)) / scale


GEOMS = [
    ("disk64", lambda: (workloads.disk(64), 2, 64, 8)),
    ("star256", lambda: (workloads.star(256), 2, 256, 8)),
    ("offdisk48_coarse6", lambda: (workloads.disk(48, 0.55, (0.13, -0.07)), 2, 48, 6)),
    ("rbox32_3d", lambda: (workloads.rounded_box(32), 3, 32, 8)),
]


@pytest.mark.parametrize("name,mk", GEOMS, ids=[g[0] for g in GEOMS])
def test_neumann_rows_match_oracle(sulfmg, oracle_mod, name, mk):
    phi, dim, N, cN = mk()
    dom, ref = _pair(sulfmg, oracle_mod, phi, dim, N, cN)
    for l in range(ref.nlev):
        gg, go = dom.level_ghosts(l), ref.level_ghosts(l)
        assert np.array_equal(gg["kind"], go["kind"])
        wg, ng_ = dom.level_rows(l)
        wo, no = ref.level_rows(l)
        _close(ng_, no, 1e-12)
        _close(wg, wo, 1e-12)
    dom.close()


RUNS = [
    ("disk64_dt_h/4", lambda: (workloads.disk(64), 2, 64, 8, 0.25 * 2.0 / 64, 5)),
    ("star256", lambda: (workloads.star(256), 2, 256, 8, 2.0 / 256, 2)),
    ("offdisk96_coarse6", lambda: (workloads.disk(96, 0.55, (0.13, -0.07)), 2, 96, 6, 0.25 * 2.0 / 96, 3)),
    ("rbox32_3d", lambda: (workloads.rounded_box(32), 3, 32, 8, 0.25 * 2.0 / 32, 2)),
]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,mk", RUNS, ids=[r[0] for r in RUNS])
def test_neumann_steps_match_oracle(sulfmg, oracle_mod, name, mk, precision):
    phi, dim, N, cN, dt, nsteps = mk()
    dom, ref = _pair(sulfmg, oracle_mod, phi, dim, N, cN)
    dom.set_solver(precision=precision)
    dom.step(dt, nsteps)
    ref.step(dt, nsteps)
    s, c, t = dom.get_state()
    rs, rc, rt = ref.get_state()
    act = (rt == 1) | (rt == 2)
    tol = RUN_TOL if precision == 0 else MIXED_TOL
    _close(s[act], rs[act], tol)
    _close(c[act], rc[act], tol)
    dom.close()


def test_switching_back_to_dirichlet_restores_the_rows(sulfmg):
    phi = workloads.star(128)
    dom = sulfmg.Domain(phi, 2, (-1.0, 1.0), 128)
    w0, _ = dom.level_rows(0)
    dom.set_bc(1)
    w1, _ = dom.level_rows(0)
    dom.set_bc(0)
    w2, _ = dom.level_rows(0)
    assert not np.array_equal(w0, w1)
    assert np.array_equal(w0, w2)
    dom.close()


LO, HI = -2.0, 2.0


def run_gpu_neumann(sulfmg, phi, N, T=1.0):
    P = workloads.PAPER_MODEL[:6]
    X, Y = workloads.node_coords(2, LO, HI, N)
    h = (HI - LO) / N
    nsteps = int(round(T / h))
    dt = T / nsteps
    dom = sulfmg.Domain(phi, 2, (LO, HI), N)
    dom.set_model(tuple(P) + (1.0, 0.0, 0.0))
    dom.set_solver(newton_tol=1e-11)
    dom.set_bc(1)
    s0, c0 = M.exact(P, X, Y, 0.0)
    dom.set_state(s0, c0, 0.0)
    B = dom.level_ghosts(0)["B"]
    _, nt = dom.level_rows(0)
    for k in range(nsteps):
        t0, t1 = k * dt, (k + 1) * dt
        f1o, f2o = M.sources(P, X, Y, t0)
        f1n, f2n = M.sources(P, X, Y, t1)
        dom.set_sources(f1o, f1n, f2o, f2n)
        dom.set_ghost_values(M.boundary_values(P, B, t1, 1, nt))
        dom.step(dt, 1)
    s, c, ty = dom.get_state()
    dom.close()
    return s, c, ty, X, Y, nsteps * dt


@pytest.mark.parametrize("test", ["test1", "test2"])
def test_neumann_accuracy_on_the_gpu(sulfmg, oracle_mod, test):
    """Tests 1N, 2N: the GPU matches the oracle driven by the same inputs at
    N = 32 and falls at second order over N = 32, 64, 128, its gradient L1
    orders within 0.3 of the paper's Tables test1sN ... test2cN."""
    P = workloads.PAPER_MODEL[:6]
    golden = json.load(open(os.path.join(HERE, "golden", "paper_accuracy_orders.json")))
    errs = {}
    for N in (32, 64, 128):
        phi = workloads.paper_test1(N) if test == "test1" else workloads.paper_test2(N)
        s, c, ty, X, Y, T = run_gpu_neumann(sulfmg, phi, N)
        if N == 32:
            rs, rc, rty, _, _, _ = M.run_oracle(oracle_mod, phi, N, LO, HI, P, bc=1)
            act = (ty == 1) | (ty == 2)
            _close(s[act], rs[act], RUN_TOL)
            _close(c[act], rc[act], RUN_TOL)
        for k, v in M.rel_errors(P, s, c, ty, X, Y, T, (HI - LO) / N).items():
            errs.setdefault(k, []).append(v)
    orders = {k: np.log2(np.array(v[:-1]) / np.array(v[1:])) for k, v in errs.items()}
    for key in ("s_1", "c_1", "gs_1", "gc_1", "s_inf", "c_inf"):
        assert orders[key].mean() >= 1.7 and orders[key].min() >= 1.3, (key, errs[key])
    for key in ("gs_1", "gc_1"):
        assert abs(orders[key].mean() - np.mean(golden[test + "N"][key])) <= 0.3, (key, errs[key])
