"""Stored-operator mode (``store_tiles``): the tensor-core apply reading
kernel values evaluated once at build.

* Per-tile store (mode 1): every tile's values exactly as the tensor core
  consumed them, so the apply equals the on-the-fly apply bit for bit.
* Symmetric store (mode 2): the real kernels are symmetric, so a block two
  tiles share is stored once and one of them reads it transposed; those
  values come from the other tile's frame and equal its own evaluation up to
  FP32 rounding. The apply matches the on-the-fly apply within the FP32
  parity tolerance (1e-5 of max |u|; measured about 1e-6).

Both match the oracle's direct sum within 10 tol.
"""
import numpy as np
import pytest
import torch

from oracle import direct
from paper_2310_16668_gb300 import SkelFMM
from paper_2310_16668_gb300 import workloads as W
from tests._util import clustered, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_16668_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("kind,dim,dist,b,tol", [("laplace3d", 3, "uniform", 64, 1e-6),
                                                 ("laplace3d", 3, "clustered", 32, 1e-6),
                                                 ("laplace2d", 2, "clustered", 32, 1e-8)])
@pytest.mark.parametrize("nrhs", [32, 64])
@pytest.mark.parametrize("mode,stages", [(1, 4), (1, 8), (1, 5), (2, 0)])
def test_stored_match_on_the_fly(kind, dim, dist, b, tol, nrhs, mode, stages):
    """Per-tile store with 4 stages per CTA (two CTAs per SM), 8 (one) and
    the split rings (5)."""
    x = W.points_uniform(20000, dim, 31) if dist == "uniform" else clustered(12000, dim, 31)
    fs = SkelFMM(x, kind, tol, b, nrhs_max=nrhs, store_tiles=mode, store_stages=stages)
    fo = SkelFMM(x, kind, tol, b, nrhs_max=nrhs)
    info = fs.info()
    assert info["store_mode"] == mode and fo.info()["store_mode"] == 0
    assert info["stored_tile_bytes"] % 16 == 0 and fo.info()["stored_tile_bytes"] == 0
    if mode == 1:
        # every tile's rows x 32 values: all kept values plus masked / ragged zeros
        assert 4 * info["pairs_tc"] <= info["stored_tile_bytes"] <= info["n_tc_tiles"] * 128 * 32 * 4
    else:
        # every distinct kept value once; shared blocks are read twice
        assert 0 < info["pairs_stored"] < info["pairs_tc"]
        assert 4 * info["pairs_stored"] <= info["stored_tile_bytes"] <= 4 * 2 * info["pairs_tc"]
    q = torch.from_numpy(W.charges_normal(x.shape[0], nrhs, 32)).cuda().float()
    us = fs.apply(q, "fp32_tc")
    uo = fo.apply(q, "fp32_tc")
    fs.device_status()
    if mode == 1:
        assert torch.equal(us, uo)
    else:
        for r in (0, nrhs // 2, nrhs - 1):
            assert relerr(us[:, r].cpu().numpy(), uo[:, r].cpu().numpy()) < 1e-5, r
        assert torch.equal(fs.apply(q, "fp32_tc"), us)    # deterministic
    ut = fs.apply_transpose(q, "fp32_tc")
    assert torch.equal(ut, us)                         # real kernels: A~^T = A~
    # and against the direct sum (RHS 0)
    ref = direct.direct_sum(kind, x, q[:, 0].double().cpu().numpy())
    assert relerr(us[:, 0].double().cpu().numpy(), ref) < 10 * tol + 1e-5


def test_stored_tiles_ignored_for_complex_kernels():
    x = clustered(3000, 3, 33)
    f = SkelFMM(x, "helmholtz3d", 1e-6, 24, kappa=25.0, store_tiles=True)
    assert f.info()["stored_tile_bytes"] == 0
    q = torch.from_numpy(W.charges_complex(x.shape[0], 1, 34)[:, 0]).cuda()
    u = f.apply(q, "fp64").cpu().numpy()
    assert relerr(u, direct.direct_sum("helmholtz3d", x, q.cpu().numpy(), kappa=25.0)) < 1e-5


@pytest.mark.slow
@pytest.mark.parametrize("mode", [1, 2])
def test_full_size_stored(mode):
    wl = W.LAPLACE3D_1M
    x = wl.make_points()
    qall = torch.from_numpy(wl.make_charges(32)).cuda().float()
    fs = SkelFMM(x, wl.kernel, wl.tol, wl.leaf, nrhs_max=32, store_tiles=mode, device_build=True)
    us = fs.apply(qall, "fp32_tc")
    fs.device_status()
    tg = wl.make_sample()
    ref = direct.direct_sum(wl.kernel, x, qall[:, 0].double().cpu().numpy(), targets=tg)
    e = relerr(us[:, 0].double().cpu().numpy()[tg], ref)
    info = fs.info()
    print(f"store mode {mode}: {info['stored_tile_bytes'] / 1e9:.1f} GB (distinct kept values "
          f"{4 * info['pairs_stored'] / 1e9:.1f} GB of {4 * info['pairs_tc'] / 1e9:.1f} GB evaluated), "
          f"device bytes {info['device_bytes'] / 1e9:.1f} GB, relerr fp32_tc {e:.3e}")
    assert e < 10 * wl.tol
    if mode == 2:
        # the symmetric store holds each shared block once
        assert info["stored_tile_bytes"] < 0.7 * 4 * info["pairs_tc"]
    fs.close()


@pytest.mark.parametrize("kind,dim", [("laplace3d", 3), ("laplace2d", 2)])
def test_autotune_keeps_results(kind, dim):
    """The autotuner only picks among variants that compute the same thing:
    the up/down launch shapes and the per-tile store give the same FP32
    result bit for bit; the symmetric store, if chosen, the on-the-fly result
    up to FP32 rounding of the shared blocks read transposed."""
    x = clustered(12000, dim, 35)
    f = SkelFMM(x, kind, 1e-6, 32, nrhs_max=32)
    q = torch.from_numpy(W.charges_normal(x.shape[0], 32, 36)).cuda().float()
    tc0, s0 = f.apply(q, "fp32_tc"), f.apply(q[:, :3].contiguous(), "fp32")
    rep = f.autotune(32, allow_store=True)
    assert rep["ms_onfly"] > 0 and rep["n_updown"] > 0
    assert rep["ms_updown_tuned"] <= rep["ms_updown_default"] + 1e-9
    assert rep["stored"] == f.info()["store_mode"]
    assert (rep["stored"] > 0) == (f.info()["stored_tile_bytes"] > 0)
    if rep["stored"] == 1:
        assert 0 < rep["ms_stored"] < rep["ms_onfly"]
    if rep["ms_stored"] > 0:
        assert rep["tcs_stages"] in (4, 5, 8)
    if rep["stored"] == 2:
        assert 0 < rep["ms_sym"] < rep["ms_onfly"]
    tc1, s1 = f.apply(q, "fp32_tc"), f.apply(q[:, :3].contiguous(), "fp32")
    f.device_status()
    assert torch.equal(s0, s1)
    if rep["stored"] == 2:
        assert relerr(tc1[:, 0].cpu().numpy(), tc0[:, 0].cpu().numpy()) < 1e-5
    else:
        assert torch.equal(tc0, tc1)
    rep2 = f.autotune(32, allow_store=False)          # tuning again is allowed
    tc2 = f.apply(q, "fp32_tc")
    if rep2["stored"] == 2:
        assert relerr(tc2[:, 0].cpu().numpy(), tc0[:, 0].cpu().numpy()) < 1e-5
    else:
        assert torch.equal(tc2, tc0)
    assert rep2["n_updown"] == rep["n_updown"]


def test_updown_launch_shapes_same_bits():
    """Every launch shape of the FP32 upward / downward passes (plain kernel
    with 1, 2, 4, 8 warps per CTA; asynchronous-copy kernel with 1, 2, 4, 8)
    gives the default's result bit for bit, in FP32 and FP32_TC, plain and
    transposed, on a deep adaptive tree with ragged boxes."""
    from paper_2310_16668_gb300 import _lib
    lib = _lib.load()
    x = clustered(12000, 3, 41)
    f = SkelFMM(x, "laplace3d", 1e-6, 16, nrhs_max=40)
    q = torch.from_numpy(W.charges_normal(x.shape[0], 40, 42)).cuda().float()
    q3 = q[:, :3].contiguous()                           # nrhs not a multiple of 4: 4-byte copies
    ref = {(p, t): (f.apply_transpose if t else f.apply)(q, p) for p in ("fp32", "fp32_tc") for t in (False, True)}
    ref3 = f.apply(q3, "fp32")
    for code in (1, 2, 4, 8, 17, 18, 20, 24):
        _lib.check(lib.skel_test_set_updown(f._h, code))
        for (p, t), r in ref.items():
            got = (f.apply_transpose if t else f.apply)(q, p)
            f.device_status()
            assert torch.equal(got, r), (code, p, t)
        assert torch.equal(f.apply(q3, "fp32"), ref3), code
    _lib.check(lib.skel_test_set_updown(f._h, 0))
