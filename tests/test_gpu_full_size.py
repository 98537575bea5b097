"""Parity at the full benchmark size, where a CN step of the oracle takes
minutes: the 257^3 rounded box (coarsest level 5^3), one CN step of the CUDA
path in the launch configuration bench.py times (default solver; FP64 and mixed
precision), then the oracle's own residual F (Eqs. FDs, FDc, BCs, evaluated by
the CPU oracle at every active node) at the GPU's state.  A converged step
solves the oracle's discrete equations: the oracle's |F|_inf at the GPU state
is as small as the GPU's own Newton residual, and the GPU's residual equals the
oracle's node by node."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbox257(oracle_mod):
    w = workloads.WORKLOADS["rbox257"]
    phi = workloads.workload_levelset("rbox257")
    ref = oracle_mod.Oracle(phi, 3, -1.0, 1.0, w["N"], w["coarsest"])
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    s0, c0, t = ref.get_state()
    return w, phi, ref, oracle_mod.interleave(s0, c0), t


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_full_size_step_solves_the_oracles_equations(sulfmg, oracle_mod, rbox257, precision):
    w, phi, ref, Wn, t = rbox257
    N = w["N"]
    dt = 2.0 / N
    dom = sulfmg.Domain(phi, 3, (-1.0, 1.0), N, w["coarsest"])
    dom.set_model(workloads.PAPER_MODEL)
    dom.set_solver(precision=precision)
    dom.step(dt, 1)
    s, c, tg = dom.get_state()
    st = dom.stats()
    assert np.array_equal(tg, t)
    W = oracle_mod.interleave(s, c)
    act = np.repeat(((t == 1) | (t == 2)).ravel(), 2)
    F_ref = ref.eval_F(dt, W, Wn)
    F_gpu = dom.eval_F(dt, W, Wn)
    dom.close()
    # the GPU's residual is the oracle's, node by node (one FP64 evaluation each)
    scale = np.abs(W[act]).max() / dt
    assert np.abs(F_gpu[act] - F_ref[act]).max() <= 1e-12 * scale
    # the converged step solves the oracle's equations to the Newton tolerance
    # (|F| of the last iterate; the step may also stop on the relative update)
    fmax = np.abs(F_ref[act]).max()
    assert fmax <= max(1e-9, 10.0 * st["last_fnorm"]), (fmax, st["last_fnorm"])
    assert fmax <= 1e-12 * scale * 1e3
