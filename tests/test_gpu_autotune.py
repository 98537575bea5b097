"""The autotuner (sulf_autotune, sulf_batch_autotune) changes only speed: the
controls it sets give the same states as the defaults (up to the summation
order of the fused coarse levels), it leaves the state untouched, and its
process cache serves same-size instances without timing."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results(sulfmg):
    N = 256
    phi = workloads.star(N)
    dt = 2.0 / N
    ref = sulfmg.Domain(phi, 2, (-1.0, 1.0), N)
    ref.set_model(workloads.PAPER_MODEL)
    ref.step(dt, 2)
    s0, c0, _ = ref.get_state()
    ref.close()
    dom = sulfmg.Domain(phi, 2, (-1.0, 1.0), N)
    dom.set_model(workloads.PAPER_MODEL)
    before = dom.get_state()
    r = dom.autotune(dt, use_cache=False)
    after = dom.get_state()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert r["candidates"] >= 8 and r["cached"] == 0
    assert 0 < r["ms_per_cycle"] <= r["ms_per_cycle_default"]
    assert r["fuse_below"] in (-1, 0, 60, 150, 400, 1000, 3000, 10000)
    dom.step(dt, 2)
    s1, c1, t = dom.get_state()
    act = (t == 1) | (t == 2)
    assert np.abs(s1[act] - s0[act]).max() <= 1e-12 * np.abs(s0[act]).max()
    assert np.abs(c1[act] - c0[act]).max() <= 1e-12 * np.abs(c0[act]).max()
    dom.close()


def test_batch_autotune_uses_the_cache(sulfmg):
    sizes = [128, 128, 256, 128]
    doms = []
    for k, N in enumerate(sizes):
        a, p, s_ext = workloads.random_star_params(np.random.default_rng(50 + k))
        d = sulfmg.Domain(workloads.random_star(N, a, p), 2, (-1.0, 1.0), N)
        m = list(workloads.PAPER_MODEL)
        m[6] = s_ext
        d.set_model(m)
        d.set_solver(precision=1)
        doms.append(d)
    b = sulfmg.Batch(doms, nstreams=2)
    res = b.autotune([2.0 / N for N in sizes])
    # the first 128 and the 256 instance are timed (unless cached earlier in
    # this process), the other 128 instances take the cached result
    assert res[1]["cached"] == 1 and res[3]["cached"] == 1
    assert res[1]["fuse_below"] == res[0]["fuse_below"]
    b.step([2.0 / N for N in sizes], 1)
    assert list(b.status()) == [0] * len(sizes)
    b.close()
    for d in doms:
        d.close()
