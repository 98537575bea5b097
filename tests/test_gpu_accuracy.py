"""The accuracy tests of Sec. 4.1 on the GPU: a manufactured solution (exact
s, c with matching sources f1, f2 and boundary values s_b at the ghosts'
boundary points) advanced to t = 1 with dt = h.  The GPU path matches the
oracle driven by the same inputs, and its errors fall at second order as in
the paper's Tables test1s/test1c/test2s/test2c (orders only: the paper's box
half-width is not given, [-2, 2] is used)."""
import json
import os

import numpy as np
import pytest

import manufactured as M
import workloads

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS = workloads.PAPER_MODEL[:6]
LO, HI = -2.0, 2.0


def run_gpu(sulfmg, phi, N, T=1.0, precision=0):
    X, Y = workloads.node_coords(2, LO, HI, N)
    h = (HI - LO) / N
    nsteps = int(round(T / h))
    dt = T / nsteps
    dom = sulfmg.Domain(phi, 2, (LO, HI), N)
    dom.set_model(tuple(PARAMS) + (1.0, 0.0, 0.0))
    dom.set_solver(newton_tol=1e-11, precision=precision)
    s0, c0 = M.exact(PARAMS, X, Y, 0.0)
    dom.set_state(s0, c0, 0.0)
    B = dom.level_ghosts(0)["B"]
    for k in range(nsteps):
        t0, t1 = k * dt, (k + 1) * dt
        f1o, f2o = M.sources(PARAMS, X, Y, t0)
        f1n, f2n = M.sources(PARAMS, X, Y, t1)
        dom.set_sources(f1o, f1n, f2o, f2n)
        sb, _ = M.exact(PARAMS, B[:, 0], B[:, 1], t1)
        dom.set_ghost_values(sb)
        dom.step(dt, 1)
    s, c, ty = dom.get_state()
    dom.close()
    return s, c, ty, X, Y, nsteps * dt


def _orders(errs):
    e = np.array(errs)
    return np.log2(e[:-1] / e[1:])


@pytest.mark.parametrize("test", ["test1", "test2"])
def test_manufactured_matches_oracle(sulfmg, oracle_mod, test):
    N = 32
    phi = workloads.paper_test1(N) if test == "test1" else workloads.paper_test2(N)
    s, c, ty, X, Y, T = run_gpu(sulfmg, phi, N)
    rs, rc, rty, _, _, _ = M.run_oracle(oracle_mod, phi, N, LO, HI, PARAMS)
    assert np.array_equal(ty, rty)
    act = (ty == 1) | (ty == 2)
    for a, b in ((s, rs), (c, rc)):
        assert np.max(np.abs(a[act] - b[act])) <= 1e-10 * np.max(np.abs(b[act]))


@pytest.mark.parametrize("test", ["test1", "test2"])
def test_second_order_on_the_gpu(sulfmg, test):
    golden = json.load(open(os.path.join(HERE, "golden", "paper_accuracy_orders.json")))
    errs = {}
    for N in (32, 64, 128):
        phi = workloads.paper_test1(N) if test == "test1" else workloads.paper_test2(N)
        s, c, ty, X, Y, T = run_gpu(sulfmg, phi, N)
        for k, v in M.rel_errors(PARAMS, s, c, ty, X, Y, T, (HI - LO) / N).items():
            errs.setdefault(k, []).append(v)
    for key in ("s_inf", "s_1", "c_inf", "c_1", "gs_1", "gc_1"):
        o = _orders(errs[key])
        assert o.mean() >= 1.8 and o.min() >= 1.6, (key, errs[key], o)
    paper = golden[test]
    for key in ("gs_1", "gc_1"):
        assert abs(_orders(errs[key]).mean() - np.mean(paper[key])) <= 0.25, (key, errs[key], paper[key])


def test_mixed_precision_keeps_the_accuracy(sulfmg):
    """FP32 cycles inside FP64 defect correction reach the same discrete
    solution: the errors against the exact solution agree with FP64's."""
    N = 64
    phi = workloads.paper_test1(N)
    e = []
    for prec in (0, 1):
        s, c, ty, X, Y, T = run_gpu(sulfmg, phi, N, precision=prec)
        e.append(M.rel_errors(PARAMS, s, c, ty, X, Y, T, (HI - LO) / N))
    for key in ("s_inf", "c_inf", "s_1", "c_1"):
        assert abs(e[1][key] - e[0][key]) <= 1e-6 * e[0][key], key
