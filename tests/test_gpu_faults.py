"""Failure detection on the GPU without a GPU fault.

* A bounded device wait that runs out: skel_test_withhold_tile makes the next
  tensor-core apply hold back one tile's copies until the compute warps have
  given up waiting for them (every wait limited to a few milliseconds). The
  apply raises the device status word (skel_device_status returns
  SKEL_ERR_TIMEOUT), nothing faults or hangs, and the next apply on the same
  plan is correct again: bit for bit the result it gave before.
* Allocation failure: skel_test_fail_alloc makes the n-th device allocation
  fail as if memory were exhausted. skel_build returns SKEL_ERR_OOM at every
  allocation it makes, frees what it had allocated (the device's free memory
  returns to where it was), and a host-pointer apply whose staging
  allocation fails returns SKEL_ERR_OOM and leaves the plan usable.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

from paper_2310_16668_gb300 import SkelFMM, _lib
from paper_2310_16668_gb300 import workloads as W
from paper_2310_16668_gb300._lib import SkelError, SkelKernel, SkelOptions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_16668_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield
    _lib.load().skel_test_fail_alloc(0)


@pytest.mark.parametrize("kind,stored,stages", [("laplace3d", 0, 0), ("laplace3d", 1, 4), ("laplace3d", 1, 5),
                                                ("laplace3d", 2, 0), ("helmholtz3d", 0, 0)])
def test_bounded_wait_runs_out(kind, stored, stages):
    """On every tensor-core kernel: on the fly, per-tile store, symmetric
    store, and the complex (3D Helmholtz) kernel."""
    x = W.points_uniform(20000, 3, 61)
    fmm = SkelFMM(x, kind, 1e-6, 64, nrhs_max=32, store_tiles=stored, store_stages=stages,
                  kappa=25.0 if kind == "helmholtz3d" else 0.0)
    assert fmm.info()["n_tc_items"] > 0 and fmm.info()["store_mode"] == stored
    if kind == "helmholtz3d":
        q = torch.from_numpy(W.charges_complex(x.shape[0], 32, 62)).cuda().to(torch.complex64)
    else:
        q = torch.from_numpy(W.charges_normal(x.shape[0], 32, 62)).cuda().float()
    ref = fmm.apply(q, "fp32_tc")
    fmm.device_status()                                          # clean before the hook
    lib = _lib.load()
    _lib.check(lib.skel_test_withhold_tile(fmm._h, 20.0))
    t0 = time.perf_counter()
    fmm.apply(q, "fp32_tc")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    with pytest.raises(SkelError) as e:
        fmm.device_status()
    assert e.value.code == -4                                    # SKEL_ERR_TIMEOUT
    assert dt < 10.0
    fmm.device_status()                                          # the word was cleared
    again = fmm.apply(q, "fp32_tc")
    fmm.device_status()
    assert torch.equal(again, ref)


def _build_rc(x, nrhs_max=8):
    lib = _lib.load()
    h = ctypes.c_void_p()
    opts = SkelOptions(0, nrhs_max, 0, 0, 0, 0)
    rc = lib.skel_build(np.ascontiguousarray(x).ctypes.data, x.shape[0], 3, SkelKernel(1, 0.0), 1e-6, 32,
                        ctypes.byref(opts), ctypes.byref(h))
    return rc, h


def test_allocation_failure_frees_everything():
    lib = _lib.load()
    x = W.points_uniform(30000, 3, 63)
    rc, h = _build_rc(x)                                         # warm-up: module loading, context
    assert rc == 0
    lib.skel_free(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for countdown in range(1, 200):
        _lib.check(lib.skel_test_fail_alloc(countdown))
        rc, h = _build_rc(x)
        if rc == 0:                                              # past the last allocation
            lib.skel_free(h)
            break
        assert rc == -2, (countdown, rc, lib.skel_last_error())
        assert h.value is None                                  # the handle is left untouched
        assert b"simulated" in lib.skel_last_error()
        failed += 1
        assert abs(torch.cuda.mem_get_info()[0] - free0) < (4 << 20), countdown
    _lib.check(lib.skel_test_fail_alloc(0))
    assert failed >= 10
    # host-pointer staging: the apply fails cleanly, the plan stays usable
    fmm = SkelFMM(x, "laplace3d", 1e-6, 32, nrhs_max=8)
    q = W.charges_normal(x.shape[0], 2, 64)
    ref = fmm.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    _lib.check(lib.skel_test_fail_alloc(1))
    with pytest.raises(SkelError) as e:
        fmm.apply(q, "fp64")                                     # numpy: staged through the plan
    assert e.value.code == -2
    _lib.check(lib.skel_test_fail_alloc(0))
    assert np.array_equal(fmm.apply(q, "fp64"), ref)
