"""skel_direct_noalloc: the direct sum for callers that cannot allocate device
memory (its partial sums live in a fixed array inside the library).

Checked through the C-ABI against the existing entry point that computes the
same sum, skel_apply on a plan whose root is a single leaf (Algorithm 2 then
reduces to the direct sum), and against the oracle's FP64 direct sum, for all
four kernels. Two calls in a row, so the second one runs on the scratch the
first left behind. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2310_16668_gb300 import SkelFMM, _lib
from paper_2310_16668_gb300 import workloads as W
from paper_2310_16668_gb300._lib import SkelKernel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_16668_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _noalloc(x, q, kind, kappa):
    lib = _lib.load()
    n, dim = x.shape
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    qd = torch.from_numpy(np.ascontiguousarray(q.T)).cuda()          # column-major n x nrhs
    ud = torch.empty_like(qd)
    stream = torch.cuda.current_stream().cuda_stream
    _lib.check(lib.skel_direct_noalloc(ctypes.c_void_p(xd.data_ptr()), n, dim,
                                       SkelKernel(_lib.KERNELS[kind], kappa), ctypes.c_void_p(qd.data_ptr()),
                                       ctypes.c_void_p(ud.data_ptr()), q.shape[1], ctypes.c_void_p(stream)))
    torch.cuda.synchronize()
    return ud.t().cpu().numpy()


@pytest.mark.parametrize("kind,dim,n", [("laplace3d", 3, 3000), ("laplace2d", 2, 2500),
                                        ("helmholtz3d", 3, 2000), ("helmholtz2d", 2, 1800)])
def test_noalloc_matches_single_leaf_apply(kind, dim, n):
    from oracle import direct
    x = W.points_uniform(n, dim, 41)
    x[7] = x[3]                                                      # a coincident pair
    cplx = kind in ("helmholtz3d", "helmholtz2d")
    q = (W.charges_complex if cplx else W.charges_normal)(n, 2, 42)
    fmm = SkelFMM(x, kind, 1e-6, n, kappa=25.0)                      # one leaf: the direct sum
    assert fmm.info()["n_levels"] == 0
    ref = fmm.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    scale = np.abs(ref).max()
    oracle = direct.direct_sum(kind, x, q, kappa=25.0)
    for _ in range(2):                                               # two calls in a row
        u = _noalloc(x, q, kind, 25.0)
        assert np.abs(u - ref).max() / scale < 1e-12
        assert np.abs(u - oracle).max() / np.abs(oracle).max() < 1e-12


@pytest.mark.parametrize("kind,dim,kappa", [("helmholtz2d", 2, 0.0), ("helmholtz2d", 2, float("nan")),
                                            ("helmholtz3d", 3, float("nan")), ("helmholtz3d", 3, -1.0)])
def test_noalloc_rejects_bad_kappa(kind, dim, kappa):
    """The kappa rules of skel_build: 2D Helmholtz needs kappa > 0, 3D Helmholtz
    kappa >= 0, both finite."""
    lib = _lib.load()
    x = torch.zeros(8 * dim, dtype=torch.float64, device="cuda")
    q = torch.zeros(16, dtype=torch.float64, device="cuda")
    u = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = lib.skel_direct_noalloc(ctypes.c_void_p(x.data_ptr()), 8, dim, SkelKernel(_lib.KERNELS[kind], kappa),
                                 ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1, None)
    assert rc == -1 and b"kappa" in lib.skel_last_error()


def test_noalloc_rejects_too_large():
    lib = _lib.load()
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    rc = lib.skel_direct_noalloc(ctypes.c_void_p(x.data_ptr()), 200000, 3, SkelKernel(1, 0.0),
                                 ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1, None)
    assert rc == -1 and b"too large" in lib.skel_last_error()
