"""The allocation-free Newton residual (sulf_newton_residual_noalloc) against
the library's own residual entry point (sulf_dbg_eval_F), through the C ABI,
on two calls in a row.

Its callers are those that cannot allocate device memory when they need a
residual (inside CUDA graph capture, or a loop that must not synchronise the
device), so its scratch is a static array in the library; two consecutive
calls check that the reused scratch gives fresh results."""
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


@pytest.mark.parametrize("dim,N", [(2, 256), (3, 32)])
def test_noalloc_residual_matches_existing_entry_point(sulfmg, dim, N):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    phi = workloads.star(N) if dim == 2 else workloads.rounded_box(N)
    dom = sulfmg.Domain(phi, dim, (-1.0, 1.0), N)
    dom.set_model(workloads.PAPER_MODEL)
    stream = torch.cuda.current_stream()
    dom.set_stream(stream.cuda_stream)
    t = dom.level_type(0)
    rng = np.random.default_rng(17)
    dt = 2.0 / N
    nn2 = 2 * t.size
    F_dev = torch.zeros(nn2, dtype=torch.float64, device="cuda")
    fnorm_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        W, act = _state(rng, t)
        Wn, _ = _state(rng, t)
        W_dev = torch.from_numpy(W).cuda()
        Wn_dev = torch.from_numpy(Wn).cuda()
        torch.cuda.synchronize()
        dom.newton_residual_noalloc(dt, W_dev.data_ptr(), Wn_dev.data_ptr(), F_dev.data_ptr(), fnorm_dev.data_ptr())
        torch.cuda.synchronize()
        F_new = F_dev.cpu().numpy()
        fnorm = float(fnorm_dev.cpu().item())
        F_ref = dom.eval_F(dt, W, Wn)
        a2 = np.repeat(act, 2)
        scale = np.abs(F_ref[a2]).max()
        assert np.abs(F_new[a2] - F_ref[a2]).max() <= TOL * scale, f"call {call}"
        assert abs(fnorm - scale) <= TOL * scale, f"call {call}"
    dom.close()
