"""Pins of the oracle's level-set preprocessing (Sec. 2): reinitialization
toward the signed distance and the provisional level set of a binary mask."""
import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("dim", [2, 3])
def test_reinit_keeps_a_plane_exactly(oracle_mod, dim):
    """A linear level set with unit gradient is a signed distance: its upwind
    differences are exact and |grad| = 1, so a step leaves every node whose
    one-sided stencil lies in the box unchanged (box-edge nodes lose the
    missing side); an axis-aligned plane, whose upwind side never leaves the
    box, is kept everywhere over many steps."""
    N = 32 if dim == 2 else 16
    C = workloads.node_coords(dim, -1.0, 1.0, N)
    nrm = np.array([0.6, -0.8] if dim == 2 else [0.48, -0.6, 0.64])
    phi = sum(nrm[a] * C[a] for a in range(dim)) - 0.1
    out = oracle_mod.reinit(phi, dim, N, 2.0 / N, 1)
    inner = (slice(1, -1),) * dim
    assert np.abs(out - phi)[inner].max() <= 1e-12
    ax = C[0] - 0.3
    assert np.abs(oracle_mod.reinit(ax, dim, N, 2.0 / N, 40) - ax).max() <= 1e-12


@pytest.mark.parametrize("N", [64, 128])
def test_reinit_turns_a_quadratic_into_the_distance(oracle_mod, N):
    """phi = |x|^2 - R^2 has the circle of radius R as zero set but |grad phi|
    = 2|x|; after 2N steps the march reaches the whole box and phi_d is the
    distance r - R to first order in h near the circle."""
    h = 2.0 / N
    X, Y = workloads.node_coords(2, -1.0, 1.0, N)
    R = 0.6
    d = oracle_mod.reinit(X * X + Y * Y - R * R, 2, N, h, 2 * N)
    r = np.sqrt(X * X + Y * Y) - R
    band = np.abs(r) < 0.3
    assert np.abs(d - r)[band].max() <= 0.5 * h
    assert np.all(np.sign(d[np.abs(r) > h]) == np.sign(r[np.abs(r) > h]))


def test_reinit_error_is_first_order(oracle_mod):
    errs = []
    for N in (32, 64, 128):
        h = 2.0 / N
        X, Y = workloads.node_coords(2, -1.0, 1.0, N)
        d = oracle_mod.reinit(0.5 * (X * X + Y * Y - 0.36), 2, N, h, 2 * N)
        r = np.sqrt(X * X + Y * Y) - 0.6
        errs.append(np.abs(d - r)[np.abs(r) < 0.25].max())
    o = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(o >= 0.7), (errs, o)


def test_mask_levelset_is_bounded_symmetric_and_has_the_right_sign(oracle_mod):
    """The heat steps keep values in [-1, 1] (maximum principle), preserve
    the mask's mirror symmetry, and leave the sign of the mask away from its
    edge; reinitialized, the zero set sits within 2 h of the mask's circle (the
    mask itself resolves the circle only to the grid)."""
    N = 64
    h = 2.0 / N
    X, Y = workloads.node_coords(2, -1.0, 1.0, N)
    R = 0.55
    mask = (X * X + Y * Y < R * R).astype(np.int8)
    ls = oracle_mod.mask_levelset(mask, 2, N, 6)
    assert ls.min() >= -1.0 and ls.max() <= 1.0
    assert np.array_equal(ls, ls[:, ::-1]) and np.array_equal(ls, ls[::-1, :])
    r = np.sqrt(X * X + Y * Y) - R
    far = np.abs(r) > 4 * h
    assert np.all(np.sign(ls[far]) == np.sign(r[far]))
    d = oracle_mod.reinit(ls, 2, N, h, 2 * N)
    assert np.abs(d - r)[np.abs(r) < 0.3].max() <= 2.0 * h


def test_mask_heat_step_keeps_linear_profiles(oracle_mod):
    """Away from the box edges one heat step maps a linear function to itself
    (the discrete Laplacian of a linear function vanishes): checked through a
    mask whose first step sees a linear +-1 profile only at its interior."""
    N = 16
    mask = np.zeros((N + 1, N + 1), dtype=np.int8)
    mask[:, : N // 2] = 1
    one = oracle_mod.mask_levelset(mask, 2, N, 1)
    # columns far from the jump and from the edges stay at -1 / +1
    assert np.all(one[:, 2: N // 2 - 2] == -1.0) and np.all(one[:, N // 2 + 2: N - 1] == 1.0)
    # the jump is smoothed symmetrically: lambda = 1/8 moves 1/4 toward each side
    assert np.allclose(one[:, N // 2 - 1], -0.75) and np.allclose(one[:, N // 2], 0.75)


def _types(phi):
    """inside phi < 0; ghost: not inside with an inside axis neighbour"""
    ins = phi < 0
    g = np.zeros_like(ins)
    for ax in range(phi.ndim):
        sl_lo = [slice(None)] * phi.ndim
        sl_hi = [slice(None)] * phi.ndim
        sl_lo[ax], sl_hi[ax] = slice(1, None), slice(None, -1)
        g[tuple(sl_lo)] |= ins[tuple(sl_hi)]
        g[tuple(sl_hi)] |= ins[tuple(sl_lo)]
    t = np.zeros(phi.shape, dtype=np.int8)
    t[ins] = 1
    t[g & ~ins] = 2
    return t


def test_extrapolation_is_exact_for_linear_data_at_a_plane(oracle_mod):
    """Linear data across a planar interface: the normal derivative is
    constant and the upwind differences are exact, so the extended values are
    the linear function itself (at ghosts away from the box edges)."""
    N = 64
    h = 2.0 / N
    X, Y = workloads.node_coords(2, -1.0, 1.0, N)
    phi = 0.6 * X - 0.8 * Y - 0.1
    t = _types(phi)
    u = 1.0 + 2.0 * X - 3.0 * Y
    e = oracle_mod.extrapolate(phi, t, u, 2, N, h, 64)
    inner = np.zeros(t.shape, dtype=bool)
    inner[4:-4, 4:-4] = True
    g = (t == 2) & inner
    assert g.sum() > 50
    assert np.abs(e - u)[g].max() <= 1e-12
    assert np.array_equal(e[t == 1], u[t == 1])


def test_extrapolation_is_second_order_at_the_ghosts(oracle_mod):
    errs = []
    for N in (32, 64, 128):
        h = 2.0 / N
        X, Y = workloads.node_coords(2, -1.0, 1.0, N)
        phi = np.sqrt(X * X + Y * Y) - 0.7
        t = _types(phi)
        u = np.sin(2 * X) * np.cos(Y) + X * Y
        e = oracle_mod.extrapolate(phi, t, u, 2, N, h, 64)
        errs.append(np.abs(e - u)[t == 2].max())
    o = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(o >= 1.8), (errs, o)
