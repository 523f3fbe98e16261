"""GPU parity: the CUDA apply (through the C-ABI) against the oracle.

* Oracle operators imported through skel_plan_import: the GPU's Algorithm 2
  must equal the oracle's Algorithm 2 element by element, to 1e-12 relative
  in FP64 and 1e-5 in FP32 (relative to max |u|), for 1 and several
  right-hand sides, the plain and the transposed apply, 2D / 3D Laplace and
  3D Helmholtz, uniform and adaptive trees (ragged boxes throughout).
* The library's own build: GPU result against the direct sum within 10 tol.
* Full size (3D Laplace, N = 2^20, leaf 128, tol 1e-6): sampled targets
  against the oracle's direct sum, in the configuration the benchmark times.
"""
import numpy as np
import pytest
import torch

from oracle import apply as oap
from oracle import direct
from oracle import plan as oplan
from oracle import skeleton as osk
from oracle import tree as otree
from paper_2310_16668_gb300 import SkelFMM, skel_apply
from paper_2310_16668_gb300 import workloads as W
from tests._util import clustered, relerr

pytestmark = pytest.mark.gpu

KAPPA = 25.0


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_16668_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _charges(kind, n, nrhs, seed):
    f = W.charges_complex if kind == "helmholtz3d" else W.charges_normal
    return f(n, nrhs, seed)


ORACLE_CASES = [
    ("laplace3d", "uniform", 6000, 24, 1e-6),
    ("laplace3d", "clustered", 5000, 20, 1e-5),
    ("laplace2d", "clustered", 6000, 16, 1e-8),
    ("helmholtz3d", "clustered", 3000, 24, 1e-6),
]


@pytest.fixture(scope="module", params=ORACLE_CASES, ids=lambda c: f"{c[0]}-{c[1]}")
def oracle_case(request):
    kind, dist, n, b, tol = request.param
    dim = 2 if kind == "laplace2d" else 3
    x = W.points_uniform(n, dim, 5) if dist == "uniform" else clustered(n, dim, 5)
    sk = osk.Skeletons(otree.Tree(x, b), kind, tol, kappa=KAPPA)
    fmm = SkelFMM.from_plan(x, kind, oplan.to_exchange(sk), kappa=KAPPA)
    return kind, x, sk, fmm


@pytest.mark.parametrize("nrhs", [1, 3])
def test_apply_matches_oracle(oracle_case, nrhs):
    kind, x, sk, fmm = oracle_case
    q = _charges(kind, x.shape[0], nrhs, 11)
    ref = oap.skeleton_apply(sk, q)
    qt = torch.from_numpy(q).cuda()
    u64 = fmm.apply(qt, "fp64").cpu().numpy()
    u32 = fmm.apply(qt, "fp32").cpu().numpy()
    utc = fmm.apply(qt, "fp32_tc").cpu().numpy()
    fmm.device_status()
    assert relerr(u64, ref) < 1e-12
    assert relerr(u32, ref) < 1e-5
    assert relerr(utc, ref) < 1e-5


@pytest.mark.parametrize("nrhs,b", [(32, 64), (45, 64), (32, 128)])
def test_tensor_core_many_rhs(nrhs, b):
    """Tensor-core translations: 45 right-hand sides = one full and one ragged
    pass; leaf size 128 puts leaves of 96..128 points (touching-leaf tasks) on
    the tensor-core path too."""
    x = W.points_uniform(40000, 3, 31)
    sk = osk.Skeletons(otree.Tree(x, b), "laplace3d", 1e-6)
    fmm = SkelFMM.from_plan(x, "laplace3d", oplan.to_exchange(sk), nrhs_max=64)
    q = W.charges_normal(x.shape[0], nrhs, 32)
    qt = torch.from_numpy(q).cuda()
    utc = fmm.apply(qt, "fp32_tc").cpu().numpy()
    fmm.device_status()
    u64 = fmm.apply(qt, "fp64").cpu().numpy()
    for r in range(nrhs):
        assert relerr(utc[:, r], u64[:, r]) < 1e-5, r
    for r in (0, nrhs - 1):
        assert relerr(u64[:, r], oap.skeleton_apply(sk, q[:, r])) < 1e-12


def test_transpose_matches_oracle(oracle_case):
    kind, x, sk, fmm = oracle_case
    q = _charges(kind, x.shape[0], 2, 12)
    ref = oap.skeleton_apply(sk, q, transpose=True)
    qt = torch.from_numpy(q).cuda()
    assert relerr(fmm.apply_transpose(qt, "fp64").cpu().numpy(), ref) < 1e-12
    assert relerr(fmm.apply_transpose(qt, "fp32").cpu().numpy(), ref) < 1e-5


def test_host_pointers_match_device(oracle_case):
    kind, x, sk, fmm = oracle_case
    q = _charges(kind, x.shape[0], 1, 13)[:, 0]
    u_host = fmm.apply(q, "fp64")                       # numpy in, numpy out: staged by the C-ABI
    u_dev = fmm.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    assert np.array_equal(u_host, u_dev)


@pytest.mark.parametrize("kind,dim,b,tol", [("laplace3d", 3, 32, 1e-6), ("laplace2d", 2, 32, 1e-8),
                                            ("helmholtz3d", 3, 32, 1e-6)])
def test_library_build_vs_direct(kind, dim, b, tol):
    x = clustered(8000, dim, 21)
    q = _charges(kind, x.shape[0], 1, 22)[:, 0]
    fmm = SkelFMM(x, kind, tol, b, kappa=KAPPA)
    ref = direct.direct_sum(kind, x, q, kappa=KAPPA)
    u = fmm.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    assert relerr(u, ref) < 10 * tol
    u32 = fmm.apply(torch.from_numpy(q).cuda(), "fp32").cpu().numpy()
    assert relerr(u32, ref) < 10 * tol + 1e-5
    utc = fmm.apply(torch.from_numpy(q).cuda(), "fp32_tc").cpu().numpy()
    fmm.device_status()
    assert relerr(utc, ref) < 10 * tol + 1e-5


@pytest.mark.parametrize("n", [1, 2, 31, 33])
def test_tiny_inputs(n):
    x = W.points_uniform(n, 3, 3)
    q = W.charges_normal(n, 1, 4)[:, 0]
    fmm = SkelFMM(x, "laplace3d", 1e-6, 16)
    u = fmm.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    ref = direct.direct_sum("laplace3d", x, q)
    if n == 1:
        assert np.all(u == 0)
    else:
        assert relerr(u, ref) < 1e-13


def test_coincident_points():
    x = W.points_uniform(2000, 3, 6)
    x[100:110] = x[5]                                   # ten copies of one point
    q = W.charges_normal(2000, 1, 7)[:, 0]
    fmm = SkelFMM(x, "laplace3d", 1e-6, 16)
    u = fmm.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    assert np.all(np.isfinite(u))
    assert relerr(u, direct.direct_sum("laplace3d", x, q)) < 1e-5


def test_autograd_laplace_gradcheck():
    x = clustered(300, 3, 8)
    fmm = SkelFMM(x, "laplace3d", 1e-6, 8)
    q = torch.from_numpy(W.charges_normal(x.shape[0], 1, 9)[:, 0]).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: skel_apply(v, fmm, "fp64"), (q,), eps=1e-6, atol=1e-8)


def test_autograd_helmholtz_backward_vs_dense():
    x = clustered(240, 3, 10)
    n = x.shape[0]
    fmm = SkelFMM(x, "helmholtz3d", 1e-6, 8, kappa=KAPPA)
    eye = torch.eye(n, dtype=torch.complex128, device="cuda")
    A = torch.stack([fmm.apply(eye[:, j].contiguous(), "fp64") for j in range(n)], dim=1)
    q = torch.from_numpy(W.charges_complex(n, 1, 11)[:, 0]).cuda().requires_grad_(True)
    w = torch.from_numpy(W.charges_complex(n, 1, 12)[:, 0]).cuda()
    loss = torch.real(torch.sum(skel_apply(q, fmm, "fp64") * w))
    loss.backward()
    # d Re(w^T A q) / d q in PyTorch's convention: conj(A^T w) ... = A^H conj(w)
    expect = (A.conj().t() @ w.conj())
    assert torch.allclose(q.grad, expect, rtol=1e-10, atol=1e-10 * expect.abs().max().item())
    # finite differences in q along a random direction
    d = torch.from_numpy(W.charges_complex(n, 1, 13)[:, 0]).cuda()
    h = 1e-6
    with torch.no_grad():
        f = lambda v: torch.real(torch.sum(fmm.apply(v, "fp64") * w))
        fd = (f(q + h * d) - f(q - h * d)) / (2 * h)
    an = torch.real(torch.sum(torch.conj(q.grad) * d))
    assert abs(fd.item() - an.item()) < 1e-6 * abs(an.item()) + 1e-9


@pytest.mark.slow
def test_full_size_laplace3d_sampled():
    wl = W.LAPLACE3D_1M
    x = wl.make_points()
    qall = wl.make_charges(32)
    q = np.ascontiguousarray(qall[:, 0])
    fmm = SkelFMM(x, wl.kernel, wl.tol, wl.leaf, nrhs_max=32)
    tg = wl.make_sample()
    ref = direct.direct_sum(wl.kernel, x, q, targets=tg)
    qt = torch.from_numpy(q).cuda()
    u64 = fmm.apply(qt, "fp64").cpu().numpy()[tg]
    u32 = fmm.apply(qt.float(), "fp32").cpu().numpy()[tg]
    utc = fmm.apply(torch.from_numpy(qall).cuda().float(), "fp32_tc").cpu().numpy()
    fmm.device_status()
    e64, e32, etc = relerr(u64, ref), relerr(u32, ref), relerr(utc[tg, 0], ref)
    print(f"full size: relerr fp64 {e64:.3e}  fp32 {e32:.3e}  fp32_tc {etc:.3e}  info {fmm.info()}")
    assert e64 < 10 * wl.tol and e32 < 10 * wl.tol and etc < 10 * wl.tol
