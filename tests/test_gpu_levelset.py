"""Level-set preprocessing of Sec. 2 on the GPU against the oracle:
reinitialization toward the signed distance, the provisional level set of a
binary mask, and a domain built from a mask stepping like the oracle."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,N", [(2, 128), (3, 32)])
def test_reinit_matches_oracle(sulfmg, oracle_mod, dim, N):
    C = workloads.node_coords(dim, -1.0, 1.0, N)
    phi = np.ascontiguousarray(sum(c * c for c in C) - 0.36)
    h = 2.0 / N
    g = sulfmg.reinit_levelset(phi, dim, N, h, 2 * N)
    o = oracle_mod.reinit(phi, dim, N, h, 2 * N)
    assert np.abs(g - o).max() <= 1e-12
    r = np.sqrt(sum(c * c for c in C)) - 0.6
    assert np.abs(g - r)[np.abs(r) < 0.25].max() <= 0.5 * h


@pytest.mark.parametrize("dim,N", [(2, 128), (3, 32)])
def test_mask_levelset_matches_oracle(sulfmg, oracle_mod, dim, N):
    C = workloads.node_coords(dim, -1.0, 1.0, N)
    mask = (sum(c * c for c in C) < 0.3).astype(np.uint8)
    g = sulfmg.levelset_from_mask(mask, dim, N, 6)
    o = oracle_mod.mask_levelset(mask.astype(np.int8), dim, N, 6)
    assert np.abs(g - o).max() <= 1e-14


def test_domain_from_a_mask_steps_like_the_oracle(sulfmg, oracle_mod):
    """A star-shaped binary mask -> provisional level set -> reinitialized
    level set -> domain: the CN steps on the GPU match the oracle's."""
    N = 128
    X, Y = workloads.node_coords(2, -1.0, 1.0, N)
    r, th = np.sqrt(X * X + Y * Y), np.arctan2(Y, X)
    mask = (r < 0.6 + 0.15 * np.sin(4 * th)).astype(np.uint8)
    h = 2.0 / N
    phi = sulfmg.reinit_levelset(sulfmg.levelset_from_mask(mask, 2, N, 4), 2, N, h, 2 * N)
    dom = sulfmg.Domain(phi, 2, (-1.0, 1.0), N)
    ref = oracle_mod.Oracle(phi, 2, -1.0, 1.0, N)
    dom.set_model(workloads.PAPER_MODEL)
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    dom.step(2.0 / N, 3)
    ref.step(2.0 / N, 3)
    s, c, t = dom.get_state()
    rs, rc, rt = ref.get_state()
    assert np.array_equal(t, rt)
    act = (rt == 1) | (rt == 2)
    for a, b in ((s, rs), (c, rc)):
        assert np.max(np.abs(a[act] - b[act])) <= 1e-10 * np.max(np.abs(b[act]))
    dom.close()


@pytest.mark.parametrize("dim,N", [(2, 64), (3, 32)])
def test_extrapolated_initial_data_match_oracle(sulfmg, oracle_mod, dim, N):
    """Non-uniform initial data given at the inside nodes: the GPU's
    extrapolated ghost values equal the oracle's extrapolation, and the CN
    steps from them match the oracle started from the same state."""
    phi = workloads.disk(N) if dim == 2 else workloads.rounded_box(N)
    C = workloads.node_coords(dim, -1.0, 1.0, N)
    s0 = 0.2 + 0.1 * np.sin(3 * C[0]) * np.cos(2 * C[1])
    c0 = 10.0 - np.cos(C[0] + C[1])
    h = 2.0 / N
    dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N)
    ref = oracle_mod.Oracle(phi, dim, -1.0, 1.0, N)
    dom.set_model(workloads.PAPER_MODEL)
    ref.set_model(workloads.PAPER_MODEL)
    ref.set_solver()
    dom.set_state_extrapolated(s0, c0, 0.0)
    s, c, t = dom.get_state()
    types = ref.level_type(0).reshape(phi.shape)
    es = oracle_mod.extrapolate(phi, types, s0, dim, N, h, 64)
    ec = oracle_mod.extrapolate(phi, types, c0, dim, N, h, 64)
    act = (types == 1) | (types == 2)
    assert np.abs(s - es)[act].max() <= 1e-12 and np.abs(c - ec)[act].max() <= 1e-12
    ins = types == 1
    assert np.array_equal(s[ins], s0[ins]) and np.array_equal(c[ins], c0[ins])
    ref.set_state(np.where(act, es, 0.0), np.where(act, ec, 0.0), 0.0)
    dt = 0.25 * h
    dom.step(dt, 2)
    ref.step(dt, 2)
    s, c, _ = dom.get_state()
    rs, rc, _ = ref.get_state()
    for a, b in ((s, rs), (c, rc)):
        assert np.max(np.abs(a[act] - b[act])) <= 1e-10 * np.max(np.abs(b[act]))
    dom.close()
