"""GPU parity at the benchmark configurations, and oracle legs for the batching
and serving runtimes.

* Star r - 0.6 - 0.2 sin 5 theta, 1025^2 nodes, dt = h, default solver
  (V(2,2), 8 levels, the coarse levels fused in one kernel): 2 CN steps.
* Rounded box ||max(|x| - 0.6, 0)||_2 - 0.2, 129^3 nodes, coarsest N = 4 (the
  3-D benchmark hierarchy), dt = h: 1 CN step.
* One instance of a batch and jobs of the server, each against the oracle
  run alone on the same inputs.

Tolerances as in the parity suite: 1e-10 relative in max-norm over the active
nodes for the FP64 form, 1e-8 for mixed precision (FP32 cycles inside FP64
defect correction)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

RUN_TOL = {0: 1e-10, 1: 1e-8}
MODEL = workloads.PAPER_MODEL


def _max_rel(a, b, act):
    return np.abs(a[act] - b[act]).max() / max(np.abs(b[act]).max(), 1e-300)


def _oracle_state(oracle_mod, phi, dim, N, cN, model, dt, nsteps):
    ref = oracle_mod.Oracle(phi, dim, -1.0, 1.0, N, cN)
    ref.set_model(model)
    ref.set_solver()
    ref.step(dt, nsteps)
    return ref.get_state()


_CACHE = {}


def _oracle_cached(oracle_mod, key, *args):
    if key not in _CACHE:
        _CACHE[key] = _oracle_state(oracle_mod, *args)
    return _CACHE[key]


CONFIGS = {
    "star1025": (lambda: workloads.star(1024), 2, 1024, 8, 2),
    "rbox129": (lambda: workloads.rounded_box(128), 3, 128, 4, 1),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_benchmark_config_matches_oracle(sulfmg, oracle_mod, name, precision):
    mk, dim, N, cN, nsteps = CONFIGS[name]
    phi = mk()
    dt = 2.0 / N
    rs, rc, rt = _oracle_cached(oracle_mod, name, phi, dim, N, cN, MODEL, dt, nsteps)
    dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N, cN)
    dom.set_model(MODEL)
    dom.set_solver(precision=precision)
    dom.step(dt, nsteps)
    s, c, t = dom.get_state()
    st = dom.stats()
    dom.close()
    assert np.array_equal(t, rt)
    act = (rt == 1) | (rt == 2)
    es, ec = _max_rel(s, rs, act), _max_rel(c, rc, act)
    assert es <= RUN_TOL[precision] and ec <= RUN_TOL[precision], (es, ec)
    assert st["steps_total"] == nsteps and st["levels"] == int(np.log2(N // cN)) + 1


def _random_star(N, seed):
    a, p, s_ext = workloads.random_star_params(np.random.default_rng(seed))
    model = list(MODEL)
    model[6] = s_ext
    return workloads.random_star(N, a, p), model


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batch_instances_match_oracle(sulfmg, oracle_mod, precision):
    sizes = [128, 512, 256, 128]
    doms, specs = [], []
    for k, N in enumerate(sizes):
        phi, model = _random_star(N, 300 + k)
        d = sulfmg.Domain(phi, 2, (-1.0, 1.0), N)
        d.set_model(model)
        d.set_solver(precision=precision)
        doms.append(d)
        specs.append((phi, N, model))
    batch = sulfmg.Batch(doms, nstreams=3)
    batch.step([2.0 / N for N in sizes], 2)
    assert list(batch.status()) == [0] * len(sizes)
    batch.close()
    for d, (phi, N, model) in zip(doms, specs):
        s, c, _ = d.get_state()
        d.close()
        if N not in (512, 256):
            continue
        rs, rc, rt = _oracle_state(oracle_mod, phi, 2, N, 8, model, 2.0 / N, 2)
        act = (rt == 1) | (rt == 2)
        assert _max_rel(s, rs, act) <= RUN_TOL[precision] and _max_rel(c, rc, act) <= RUN_TOL[precision]


def test_server_jobs_match_oracle(sulfmg, oracle_mod):
    jobs = []
    for k, N in enumerate([256, 512, 128]):
        phi, model = _random_star(N, 400 + k)
        jobs.append(dict(phi=phi, dim=2, N=N, cN=8, model=model, dt=2.0 / N, nsteps=2, precision=k % 2))
    phi3, _, _ = workloads.random_rounded_box(64, np.random.default_rng(7))
    jobs.append(dict(phi=phi3, dim=3, N=64, cN=4, model=list(MODEL), dt=0.25 * 2.0 / 64, nsteps=2, precision=1))
    srv = sulfmg.Server(budget_bytes=40 << 30, nworkers=3)
    ids = [srv.submit(j["phi"], j["dim"], j["N"], j["model"], j["dt"], j["nsteps"], coarsest_N=j["cN"],
                      precision=j["precision"]) for j in jobs]
    out = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for j, (s, c, res) in zip(jobs, out):
        rs, rc, rt = _oracle_state(oracle_mod, j["phi"], j["dim"], j["N"], j["cN"], j["model"], j["dt"], j["nsteps"])
        act = (rt == 1) | (rt == 2)
        s = s.reshape(rs.shape)
        c = c.reshape(rc.shape)
        tol = RUN_TOL[j["precision"]]
        assert _max_rel(s, rs, act) <= tol and _max_rel(c, rc, act) <= tol, (j["dim"], j["N"])
