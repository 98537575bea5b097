"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h; argument errors are reported without touching a GPU."""
import ctypes
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in ("sulfmg.h", "sulfmg_debug.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(sulf_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(sulfmg):
    lib = sulfmg.load()
    names = _declared()
    assert len(names) >= 20
    missing = sorted(n for n in names if not hasattr(lib, n))
    assert not missing, missing


def test_binding_covers_the_abi(sulfmg):
    bound = set(sulfmg._SIGS)
    assert _declared() == bound


def test_argument_errors_without_gpu(sulfmg):
    lib = sulfmg.load()
    phi = np.ones(17 * 17)
    box = np.array([-1.0, 1.0])
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    # N = 12 is not coarsest_N * 2^k for coarsest_N = 8
    rc = lib.sulf_create_domain(phi.ctypes.data_as(dp), 2, box.ctypes.data_as(dp), 12, 8, ctypes.byref(h))
    assert rc == sulfmg.EINVAL and not h.value
    assert b"power of two" in lib.sulf_last_error()
    rc = lib.sulf_create_domain(phi.ctypes.data_as(dp), 4, box.ctypes.data_as(dp), 16, 8, ctypes.byref(h))
    assert rc == sulfmg.EINVAL
    rc = lib.sulf_create_domain(None, 2, box.ctypes.data_as(dp), 16, 8, ctypes.byref(h))
    assert rc == sulfmg.EINVAL
    assert lib.sulf_step(None, 0.1, 1) == sulfmg.EINVAL
    out = np.zeros(17 * 17)
    assert lib.sulf_reinit_levelset(None, 2, 16, 0.1, 4, out.ctypes.data_as(dp)) == sulfmg.EINVAL
    assert lib.sulf_reinit_levelset(phi.ctypes.data_as(dp), 4, 16, 0.1, 4, out.ctypes.data_as(dp)) == sulfmg.EINVAL
    assert lib.sulf_levelset_from_mask(None, 2, 16, 4, out.ctypes.data_as(dp)) == sulfmg.EINVAL
    assert lib.sulf_set_bc(None, 1) == sulfmg.EINVAL
    assert lib.sulf_set_solver(None, None) == sulfmg.EINVAL
    # batching: a NULL batch or bad arguments are refused before any device work
    assert lib.sulf_batch_set_lockstep(None, 1) == sulfmg.EINVAL
    assert lib.sulf_batch_step(None, None, None) == sulfmg.EINVAL
    assert lib.sulf_batch_autotune(None, None, None) == sulfmg.EINVAL
    assert lib.sulf_batch_status(None, None) == sulfmg.EINVAL
    b = ctypes.c_void_p()
    assert lib.sulf_batch_create(None, 2, 1, ctypes.byref(b)) == sulfmg.EINVAL and not b.value
    lib.sulf_destroy(None)


def test_headers_cite_the_paper():
    for h in ("sulfmg.h", "sulfmg_debug.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        assert "arXiv:1902.07029" in src or "Sec. 3" in src


def test_memory_estimate_host_logic(sulfmg):
    est = sulfmg.estimate_device_bytes
    assert est(2, 0, 8, 0) == 0 and est(4, 64, 8, 0) == 0
    assert est(2, 128, 8, 0) < est(2, 256, 8, 0) < est(2, 512, 8, 0)
    assert est(2, 256, 8, 0) < est(2, 256, 8, 1)
    assert est(3, 64, 8, 0) > est(2, 64, 8, 0)
