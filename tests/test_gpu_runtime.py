"""Batching and serving: every instance's result in a batch or in the server's
mix equals its result computed alone (bit for bit: the kernels are
deterministic), admission keeps the reserved device memory within the budget,
and a failing job does not disturb the others."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

MODEL = workloads.PAPER_MODEL


def _random_star(N, seed):
    a, p, s_ext = workloads.random_star_params(np.random.default_rng(seed))
    model = list(MODEL)
    model[6] = s_ext
    return workloads.random_star(N, a, p), model


def _alone(sulfmg, phi, dim, N, model, dt, nsteps, **solver):
    dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N)
    dom.set_model(model)
    dom.set_solver(**solver)
    dom.step(dt, nsteps)
    s, c, _ = dom.get_state()
    dom.close()
    return s, c


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_instances_alone(sulfmg, precision):
    sizes = [128, 256, 128, 512, 256, 128]
    doms, specs = [], []
    for k, N in enumerate(sizes):
        phi, model = _random_star(N, 100 + k)
        d = sulfmg.Domain(phi, 2, (-1.0, 1.0), N)
        d.set_model(model)
        d.set_solver(precision=precision)
        doms.append(d)
        specs.append((phi, N, model))
    batch = sulfmg.Batch(doms, nstreams=3)
    dts = [2.0 / N for N in sizes]
    # two calls: between them instances move to whichever worker stream is free
    batch.step(dts, 1)
    batch.step(dts, 1)
    assert list(batch.status()) == [0] * len(sizes)
    batch.close()
    for d, (phi, N, model) in zip(doms, specs):
        s, c, _ = d.get_state()
        s1, c1 = _alone(sulfmg, phi, 2, N, model, 2.0 / N, 2, precision=precision)
        assert np.array_equal(s, s1) and np.array_equal(c, c1)
        d.close()


def _jobs():
    jobs = []
    for k, N in enumerate([256, 128, 512, 128, 256]):
        phi, model = _random_star(N, 200 + k)
        jobs.append(dict(levelset=phi, dim=2, N=N, model=model, dt=2.0 / N, nsteps=1 + k % 3,
                         precision=k % 2))
    jobs.append(dict(levelset=workloads.rounded_box(32), dim=3, N=32, model=list(MODEL), dt=0.25 * 2.0 / 32,
                     nsteps=1, precision=0))
    return jobs


def test_server_results_same_alone_and_in_the_mix(sulfmg):
    jobs = _jobs()
    srv = sulfmg.Server(budget_bytes=40 << 30, nworkers=3)
    ids = [srv.submit(j["levelset"], j["dim"], j["N"], j["model"], j["dt"], j["nsteps"], precision=j["precision"])
           for j in jobs]
    out = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["max_running"] >= 2, "jobs did not overlap on the device"
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for j, (s, c, res) in zip(jobs, out):
        s1, c1 = _alone(sulfmg, j["levelset"], j["dim"], j["N"], j["model"], j["dt"], j["nsteps"],
                        precision=j["precision"])
        assert np.array_equal(s, s1) and np.array_equal(c, c1)
        assert res["device_bytes"] <= res["estimate_bytes"]


def test_server_admission_respects_budget(sulfmg):
    N = 256
    est = sulfmg.estimate_device_bytes(2, N, 8, 0)
    budget = int(2.5 * est)
    srv = sulfmg.Server(budget_bytes=budget, nworkers=4)
    ids = []
    for k in range(6):
        phi, model = _random_star(N, 300 + k)
        ids.append(srv.submit(phi, 2, N, model, 2.0 / N, 2))
    for i in ids:
        srv.wait(i)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 6
    assert st["peak_reserved_bytes"] <= budget
    assert st["max_running"] <= 2
    with pytest.raises(sulfmg.SulfError) as e:
        small = sulfmg.Server(budget_bytes=est // 2, nworkers=1)
        try:
            small.submit(workloads.star(N), 2, N, list(MODEL), 2.0 / N, 1)
        finally:
            small.close()
    assert e.value.code == sulfmg.ENOMEM


def test_server_failing_job_is_isolated(sulfmg):
    """65^2 disk with dt = h has no discrete solution at its second step (the
    CN c-equation of some ghosts has no real root): Newton reports ENOTCONV for
    that job only."""
    srv = sulfmg.Server(budget_bytes=16 << 30, nworkers=2)
    good_phi, model = _random_star(128, 400)
    g1 = srv.submit(good_phi, 2, 128, model, 2.0 / 128, 2)
    bad = srv.submit(workloads.disk(64), 2, 64, list(MODEL), 2.0 / 64, 10)
    g2 = srv.submit(good_phi, 2, 128, model, 2.0 / 128, 2)
    s1, c1, _ = srv.wait(g1)
    with pytest.raises(sulfmg.SulfError) as e:
        srv.wait(bad)
    assert e.value.code == sulfmg.ENOTCONV
    s2, c2, _ = srv.wait(g2)
    st = srv.stats()
    srv.close()
    assert st["failed"] == 1 and st["completed"] == 2
    assert np.array_equal(s1, s2) and np.array_equal(c1, c2)


@pytest.mark.parametrize("dim,N,precision", [(2, 128, 0), (2, 512, 1), (3, 32, 0), (3, 64, 1)])
def test_estimate_covers_the_allocation(sulfmg, dim, N, precision):
    phi = workloads.star(N) if dim == 2 else workloads.rounded_box(N)
    dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N)
    dom.set_model(MODEL)
    dom.set_solver(precision=precision)
    dom.step(0.25 * 2.0 / N, 1)
    used = dom.stats()["device_bytes"]
    dom.close()
    assert used <= sulfmg.estimate_device_bytes(dim, N, 8, precision)
