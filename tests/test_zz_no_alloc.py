"""The allocation-free Newton residual (sulf_newton_residual_noalloc) through
the C ABI, on two calls in a row.

It serves callers that cannot allocate device memory when they need a
residual: an application whose own memory manager has already reserved the
device memory it may use, or a time-critical loop that must not take the
device-wide synchronisation of a cudaMalloc/cudaFree.  Its scratch is therefore
a static array inside the library that every call reuses; two consecutive calls
on fresh inputs check that the reused scratch gives fresh results.  The output
is compared with the library's existing residual entry point (sulf_dbg_eval_F)
and with the CPU oracle's F, and the documented refusals (misaligned pointers,
Neumann rows) are checked without launching anything.

This file is collected last on purpose: a failure here leaves every other test
already run."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12  # one kernel application, rounding order only (as the stage parity tests)


def _state(rng, t):
    act = (t == 1) | (t == 2)
    W = np.zeros(2 * t.size)
    W[0::2][act] = rng.uniform(0.0, 1.0, act.sum())
    W[1::2][act] = rng.uniform(5.0, 10.0, act.sum())
    return W, act


def _domain(sulfmg, torch, dim, N):
    phi = workloads.star(N) if dim == 2 else workloads.rounded_box(N)
    dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N)
    dom.set_model(workloads.PAPER_MODEL)
    dom.set_stream(torch.cuda.current_stream().cuda_stream)
    return phi, dom


@pytest.mark.parametrize("dim,N", [(2, 256), (3, 32)])
def test_noalloc_residual_matches_existing_entry_point_and_oracle(sulfmg, oracle_mod, dim, N):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    phi, dom = _domain(sulfmg, torch, dim, N)
    ref = oracle_mod.Oracle(phi, dim, -1.0, 1.0, N)
    ref.set_model(workloads.PAPER_MODEL)
    t = dom.level_type(0)
    rt = ref.level_type(0)
    assert np.array_equal((t == 1) | (t == 2), (rt == 1) | (rt == 2))
    rng = np.random.default_rng(17)
    dt = 2.0 / N
    nn2 = 2 * t.size
    # every buffer the calls touch exists before the first call
    F_dev = torch.zeros(nn2, dtype=torch.float64, device="cuda")
    fnorm_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    W_dev = torch.zeros(nn2, dtype=torch.float64, device="cuda")
    Wn_dev = torch.zeros(nn2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for call in range(2):
        W, act = _state(rng, t)
        Wn, _ = _state(rng, t)
        W_dev.copy_(torch.from_numpy(W))
        Wn_dev.copy_(torch.from_numpy(Wn))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        dom.newton_residual_noalloc(dt, W_dev.data_ptr(), Wn_dev.data_ptr(), F_dev.data_ptr(), fnorm_dev.data_ptr())
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, f"call {call} changed the free device memory"
        F_new = F_dev.cpu().numpy()
        fnorm = float(fnorm_dev.cpu().item())
        a2 = np.repeat(act, 2)
        for label, F_ref in (("library", dom.eval_F(dt, W, Wn)), ("oracle", ref.eval_F(dt, W, Wn))):
            scale = np.abs(F_ref[a2]).max()
            assert np.abs(F_new[a2] - F_ref[a2]).max() <= TOL * scale, f"call {call} vs {label}"
            assert abs(fnorm - scale) <= TOL * scale, f"call {call} norm vs {label}"
    dom.close()


def test_noalloc_residual_refusals(sulfmg):
    """Misaligned buffers and Neumann rows are refused on the host with
    SULF_EINVAL, before anything is queued; the handle stays usable."""
    torch = pytest.importorskip("torch")
    N = 64
    _, dom = _domain(sulfmg, torch, 2, N)
    nn2 = 2 * (N + 1) ** 2
    buf = torch.zeros(4 * nn2 + 8, dtype=torch.float64, device="cuda")
    base = buf.data_ptr()
    W, Wn, F, fn = base, base + 8 * nn2, base + 16 * nn2, base + 8 * (4 * nn2)
    dt = 2.0 / N
    for args in ((W + 8, Wn, F, fn), (W, Wn + 8, F, fn), (W, Wn, F + 8, fn), (W, Wn, F, fn + 4)):
        with pytest.raises(sulfmg.SulfError) as e:
            dom.newton_residual_noalloc(dt, *args)
        assert e.value.code == sulfmg.EINVAL and "aligned" in str(e.value)
    dom.set_bc(1)
    with pytest.raises(sulfmg.SulfError) as e:
        dom.newton_residual_noalloc(dt, W, Wn, F, fn)
    assert e.value.code == sulfmg.EINVAL
    dom.set_bc(0)
    dom.newton_residual_noalloc(dt, W, Wn, F, fn)
    torch.cuda.synchronize()
    dom.close()
