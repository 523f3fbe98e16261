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
    f = W.charges_complex if kind in ("helmholtz3d", "helmholtz2d") else W.charges_normal
    return f(n, nrhs, seed)


ORACLE_CASES = [
    ("laplace3d", "uniform", 6000, 24, 1e-6),
    ("laplace3d", "clustered", 5000, 20, 1e-5),
    ("laplace2d", "clustered", 6000, 16, 1e-8),
    ("helmholtz3d", "clustered", 3000, 24, 1e-6),
    ("helmholtz2d", "clustered", 3000, 16, 1e-8),
]


@pytest.fixture(scope="module", params=ORACLE_CASES, ids=lambda c: f"{c[0]}-{c[1]}")
def oracle_case(request):
    kind, dist, n, b, tol = request.param
    dim = 2 if kind in ("laplace2d", "helmholtz2d") else 3
    x = W.points_uniform(n, dim, 5) if dist == "uniform" else clustered(n, dim, 5)
    sk = osk.Skeletons(otree.Tree(x, b), kind, tol, kappa=KAPPA)
    fmm = SkelFMM.from_plan(x, kind, oplan.to_exchange(sk), kappa=KAPPA)
    return kind, x, sk, fmm


@pytest.mark.parametrize("nrhs", [1, 3, 4])
def test_apply_matches_oracle(oracle_case, nrhs):
    """nrhs = 4 puts the real kernels' FP32_TC apply on the tensor cores."""
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


@pytest.mark.parametrize("nrhs,b", [(16, 64), (21, 64), (16, 128)])
def test_tensor_core_helmholtz_many_rhs(nrhs, b):
    """Complex tensor-core translations (3D Helmholtz, kappa = 25): 21
    right-hand sides = one full pass of 16 and a ragged one; leaf size 128
    puts touching leaves (coincident-free close pairs) on the tensor cores.
    Every column against the FP64 apply, and the transposed apply."""
    x = W.points_uniform(30000, 3, 33)
    sk = osk.Skeletons(otree.Tree(x, b), "helmholtz3d", 1e-6, kappa=KAPPA)
    fmm = SkelFMM.from_plan(x, "helmholtz3d", oplan.to_exchange(sk), kappa=KAPPA, nrhs_max=32)
    assert fmm.info()["n_tc_items"] > 0
    q = W.charges_complex(x.shape[0], nrhs, 34)
    qt = torch.from_numpy(q).cuda()
    utc = fmm.apply(qt.to(torch.complex64), "fp32_tc").cpu().numpy()
    fmm.device_status()
    u64 = fmm.apply(qt, "fp64").cpu().numpy()
    for r in range(nrhs):
        assert relerr(utc[:, r], u64[:, r]) < 1e-5, r
    assert relerr(u64[:, nrhs - 1], oap.skeleton_apply(sk, q[:, nrhs - 1])) < 1e-12
    vtc = fmm.apply_transpose(qt.to(torch.complex64), "fp32_tc").cpu().numpy()
    v64 = fmm.apply_transpose(qt, "fp64").cpu().numpy()
    for r in (0, nrhs - 1):
        assert relerr(vtc[:, r], v64[:, r]) < 1e-5, r


@pytest.mark.parametrize("updown_tc", [False, True])
def test_tensor_core_updown_accuracy(updown_tc):
    """FP32_TC on a deep tree (five levels, items of two row blocks, inner
    sizes up to 1,200), with the upward / downward skeleton GEMMs on the CUDA
    cores (default) or on the tensor cores (skel_options.updown_tc): every
    column within 2e-6 of the FP64 apply (the FP32 CUDA-core apply: about
    2e-7), and the transposed apply too."""
    x = W.points_uniform(150000, 3, 37)
    fmm = SkelFMM(x, "laplace3d", 1e-6, 32, nrhs_max=32, updown_tc=updown_tc)
    q = torch.from_numpy(W.charges_normal(x.shape[0], 32, 38)).cuda()
    u64 = fmm.apply(q, "fp64").cpu().numpy()
    utc = fmm.apply(q.float(), "fp32_tc").cpu().numpy()
    u32 = fmm.apply(q[:, :2].float().contiguous(), "fp32").cpu().numpy()
    fmm.device_status()
    e32 = max(relerr(u32[:, r], u64[:, r]) for r in range(2))
    etc = max(relerr(utc[:, r], u64[:, r]) for r in range(32))
    print(f"updown_tc {updown_tc}: fp32 vs fp64 {e32:.2e}, fp32_tc vs fp64 {etc:.2e}")
    assert etc < 2e-6
    vtc = fmm.apply_transpose(q.float(), "fp32_tc").cpu().numpy()
    assert max(relerr(vtc[:, r], u64[:, r]) for r in (0, 31)) < 2e-6   # Laplace: A~^T = A~


def test_transpose_matches_oracle(oracle_case):
    kind, x, sk, fmm = oracle_case
    q = _charges(kind, x.shape[0], 4, 12)
    ref = oap.skeleton_apply(sk, q, transpose=True)
    qt = torch.from_numpy(q).cuda()
    assert relerr(fmm.apply_transpose(qt, "fp64").cpu().numpy(), ref) < 1e-12
    assert relerr(fmm.apply_transpose(qt, "fp32").cpu().numpy(), ref) < 1e-5
    assert relerr(fmm.apply_transpose(qt, "fp32_tc").cpu().numpy(), ref) < 1e-5


def test_host_pointers_match_device(oracle_case):
    """Host buffers give the device result bit for bit: pageable ones are
    staged by the C-ABI, page-locked ones read and written in place by the
    permutation kernels (1 and 32 right-hand sides: both permutation forms)."""
    kind, x, sk, fmm = oracle_case
    q = _charges(kind, x.shape[0], 1, 13)[:, 0]
    u_host = fmm.apply(q, "fp64")                       # numpy in, numpy out: staged by the C-ABI
    u_dev = fmm.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    assert np.array_equal(u_host, u_dev)
    for nrhs in (1, 32):
        qn = torch.from_numpy(np.ascontiguousarray(_charges(kind, x.shape[0], nrhs, 14).T))
        qp = qn.pin_memory()
        up = torch.empty_like(qp).pin_memory()
        fmm.apply_into(qp.t(), up.t(), nrhs, "fp64")
        ud = torch.empty_like(qn).cuda()
        fmm.apply_into(qn.cuda().t(), ud.t(), nrhs, "fp64")
        torch.cuda.synchronize()
        assert torch.equal(up, ud.cpu())


@pytest.mark.parametrize("kind,dim,b,tol", [("laplace3d", 3, 32, 1e-6), ("laplace2d", 2, 32, 1e-8),
                                            ("helmholtz3d", 3, 32, 1e-6), ("helmholtz2d", 2, 32, 1e-8)])
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
    e64, e32 = relerr(u64, ref), relerr(u32, ref)
    # the tensor-core pass: its first, an inner and its last B-operand column
    etc = {}
    for r in (0, 17, 31):
        ref_r = ref if r == 0 else direct.direct_sum(wl.kernel, x, np.ascontiguousarray(qall[:, r]), targets=tg)
        etc[r] = relerr(utc[tg, r], ref_r)
    print(f"full size: relerr fp64 {e64:.3e}  fp32 {e32:.3e}  fp32_tc {etc}  info {fmm.info()}")
    assert e64 < 10 * wl.tol and e32 < 10 * wl.tol and max(etc.values()) < 10 * wl.tol


@pytest.mark.slow
def test_full_size_sphere_cluster_sampled():
    """Adaptive 3D Laplace, N = 2^22 on the unit sphere plus a Gaussian cluster
    (a deep tree with coarse and fine neighbors), 32 right-hand sides on the
    tensor-core path: sampled targets against the oracle's direct sum."""
    wl = W.LAPLACE3D_ADAPTIVE_4M
    x = wl.make_points()
    qall = wl.make_charges(32)
    fmm = SkelFMM(x, wl.kernel, wl.tol, wl.leaf, nrhs_max=32)
    info = fmm.info()
    assert info["n_coarse"] > 0 and info["n_fine"] > 0
    tg = wl.make_sample()
    utc = fmm.apply(torch.from_numpy(qall).cuda().float(), "fp32_tc").cpu().numpy()
    fmm.device_status()
    for r in (0, 31):
        ref = direct.direct_sum(wl.kernel, x, np.ascontiguousarray(qall[:, r]), targets=tg)
        e = relerr(utc[tg, r], ref)
        print(f"sphere+cluster: RHS {r} relerr {e:.3e}  levels {info['n_levels']}")
        assert e < 10 * wl.tol


@pytest.mark.slow
def test_full_size_helmholtz_sampled():
    """3D Helmholtz (kappa = 25), N = 2^20: complex128, complex64 and the
    complex64 tensor-core applies at sampled targets against the oracle's
    complex128 direct sum."""
    wl = W.HELMHOLTZ3D_1M
    x = wl.make_points()
    q = wl.make_charges(4)
    fmm = SkelFMM(x, wl.kernel, wl.tol, wl.leaf, kappa=wl.kappa, nrhs_max=4)
    tg = wl.make_sample()[:1024]
    ref = direct.direct_sum(wl.kernel, x, np.ascontiguousarray(q[:, 1]), targets=tg, kappa=wl.kappa)
    qt = torch.from_numpy(q).cuda()
    u64 = fmm.apply(qt, "fp64").cpu().numpy()[tg, 1]
    u32 = fmm.apply(qt.to(torch.complex64), "fp32").cpu().numpy()[tg, 1]
    utc = fmm.apply(qt.to(torch.complex64), "fp32_tc").cpu().numpy()[tg, 1]
    fmm.device_status()
    e64, e32, etc = relerr(u64, ref), relerr(u32, ref), relerr(utc, ref)
    print(f"helmholtz: relerr complex128 {e64:.3e} complex64 {e32:.3e} complex64 tensor cores {etc:.3e}")
    assert e64 < 10 * wl.tol and e32 < 10 * wl.tol and etc < 10 * wl.tol


def test_helmholtz2d_fp32_kernel_values():
    """The FP32 2D Helmholtz kernel value by value, through the C-ABI: on a
    single-leaf plan the apply is the direct sum, so unit charges return the
    kernel matrix column by column. kappa = 100 and distances from 1e-6 to
    1.41 put kappa r on both sides of 8 (the library's series / asymptotic
    switch) up to 141; compared with the oracle's complex128 kernel (the
    Bessel functions of scipy) relative to |G|."""
    from oracle import kernels
    n, kappa = 64, 100.0
    t = np.concatenate([[0.0], np.geomspace(1e-6, 1.42, n - 1)])
    th = np.linspace(0.0, 0.7, n)
    x = np.stack([0.01 + t * np.cos(0.785 + 0.05 * th), 0.005 + t * np.sin(0.785 + 0.05 * th)], axis=1)
    fmm = SkelFMM(x, "helmholtz2d", 1e-6, n, kappa=kappa, nrhs_max=n)
    assert fmm.info()["n_levels"] == 0
    G = fmm.apply(torch.eye(n, dtype=torch.complex64, device="cuda"), "fp32").cpu().numpy()
    ref = kernels.kernel_matrix("helmholtz2d", x, x, kappa)
    off = ~np.eye(n, dtype=bool)
    kr = kappa * np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
    assert kr[off].min() < 1e-3 and kr.max() > 140 and np.any((kr > 8) & (kr < 20))
    err = np.abs(G - ref)[off] / np.abs(ref)[off]
    assert np.all(np.diag(G) == 0)
    assert err.max() < 2e-6, (err.max(), kr[off][np.argmax(err)])


@pytest.mark.slow
def test_full_size_helmholtz2d_sampled():
    """2D Helmholtz (kappa = 100, about 16 wavelengths across the square),
    N = 2^20, leaf 64, tol 1e-6: complex64 and complex128 applies at 4096
    sampled targets against the oracle's complex128 direct sum, within
    10 tol (the FP32 path carries the phase kappa r as a double-float)."""
    wl = W.HELMHOLTZ2D_1M
    x = wl.make_points()
    q = wl.make_charges(2)
    fmm = SkelFMM(x, wl.kernel, wl.tol, wl.leaf, kappa=wl.kappa, nrhs_max=2)
    tg = wl.make_sample()
    ref = direct.direct_sum(wl.kernel, x, np.ascontiguousarray(q[:, 0]), targets=tg, kappa=wl.kappa)
    qt = torch.from_numpy(q).cuda()
    u64 = fmm.apply(qt, "fp64").cpu().numpy()[tg, 0]
    u32 = fmm.apply(qt.to(torch.complex64), "fp32").cpu().numpy()[tg, 0]
    fmm.device_status()
    e64, e32 = relerr(u64, ref), relerr(u32, ref)
    print(f"helmholtz2d: relerr complex128 {e64:.3e} complex64 {e32:.3e}")
    assert e64 < 10 * wl.tol and e32 < 10 * wl.tol


def test_batched_curve_sets_and_graph():
    """Several independent 2D point sets on closed curves: the batched apply
    equals each set's own apply, matches the oracle's direct sum within
    10 tol, and a CUDA graph of the batch plus its adjoint replays to the
    same result."""
    from paper_2310_16668_gb300 import SkelBatch
    cs = W.CurveSets(n_sets=6, seed=21)
    sets = [W.points_curve(n, 900 + i) for i, n in enumerate((700, 1500, 2600, 1100, 3300, 900))]
    nrhs = 4
    b = SkelBatch(sets, "laplace2d", cs.tol, 16, nrhs_max=nrhs)
    qs = [torch.from_numpy(np.ascontiguousarray(cs.make_charges(i, len(x), nrhs).T)).cuda().float()
          for i, x in enumerate(sets)]
    us = [torch.empty_like(q) for q in qs]
    b.apply_into(qs, us, nrhs, "fp32_tc")
    torch.cuda.synchronize()
    for i, (f, x) in enumerate(zip(b.plans, sets)):
        one = torch.empty_like(qs[i])
        f.apply_into(qs[i], one, nrhs, "fp32_tc")
        torch.cuda.synchronize()
        assert torch.equal(one, us[i])                        # same kernels, same order
        ref = direct.direct_sum("laplace2d", x, qs[i][2].double().cpu().numpy())
        u64 = torch.empty_like(qs[i], dtype=torch.float64)
        f.apply_into(qs[i].double(), u64, nrhs, "fp64")
        torch.cuda.synchronize()
        e64, etc = relerr(u64[2].cpu().numpy(), ref), relerr(us[i][2].double().cpu().numpy(), ref)
        print(f"curve set {i} (n = {len(x)}): relerr fp64 {e64:.2e} fp32_tc {etc:.2e}")
        assert e64 < 10 * cs.tol and etc < 10 * cs.tol
    # graph: forward batch + adjoint batch, replayed on fresh inputs
    gs = [torch.randn_like(q) for q in qs]
    vs = [torch.empty_like(q) for q in qs]
    g = b.capture(qs, us, nrhs, "fp32_tc", adjoint_qs=gs, adjoint_us=vs)
    for q in qs:
        q.mul_(-2.0)
    g.replay()
    torch.cuda.synchronize()
    for i, f in enumerate(b.plans):
        e1, e2 = torch.empty_like(qs[i]), torch.empty_like(gs[i])
        f.apply_into(qs[i], e1, nrhs, "fp32_tc")
        f.apply_into(gs[i], e2, nrhs, "fp32_tc", transpose=True)
        torch.cuda.synchronize()
        assert torch.equal(e1, us[i]) and torch.equal(e2, vs[i])
    b.close()


def test_merged_plan_equals_per_set_applies():
    """skel_merge: one plan over several independent curve sets applies every
    set in one pass (one launch per phase over all sets) and gives each set
    exactly its own apply's values, for every precision and the transpose;
    a CUDA graph of the merged forward and adjoint replays to the same."""
    from paper_2310_16668_gb300 import SkelBatch
    cs = W.CurveSets(n_sets=6, seed=21)
    sets = [W.points_curve(n, 900 + i) for i, n in enumerate((700, 1500, 2600, 1100, 3300, 900))]
    nrhs = 4
    b = SkelBatch(sets, "laplace2d", cs.tol, 16, nrhs_max=nrhs)
    m = b.merged()
    assert m.n == sum(b.sizes)
    off = b.offsets
    for prec in ("fp64", "fp32", "fp32_tc"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        qs = [torch.from_numpy(np.ascontiguousarray(cs.make_charges(i, len(x), nrhs).T)).cuda().to(dt)
              for i, x in enumerate(sets)]
        Q = torch.cat(qs, dim=1).contiguous()                   # (nrhs, N): N x nrhs column-major
        for transpose in (False, True):
            U = torch.empty_like(Q)
            m.set_profiling(1)
            m.apply_into(Q, U, nrhs, prec, transpose=transpose)
            merged_launches = m.last_timings()["launches"]
            m.set_profiling(0)
            m.device_status()
            per_set = []
            for i, f in enumerate(b.plans):
                one = torch.empty_like(qs[i])
                f.set_profiling(1)
                f.apply_into(qs[i], one, nrhs, prec, transpose=transpose)
                per_set.append(f.last_timings()["launches"])
                f.set_profiling(0)
                torch.cuda.synchronize()
                assert torch.equal(one, U[:, off[i]:off[i + 1]]), (prec, transpose, i)
            # one launch per phase (and level) over all sets: as many as the
            # deepest set's own apply, not the sum over the sets
            assert merged_launches <= max(per_set) + 2 < sum(per_set), (merged_launches, per_set)
    # graph of the merged forward and adjoint, replayed on new inputs
    Q = torch.cat([torch.from_numpy(np.ascontiguousarray(cs.make_charges(i, len(x), nrhs).T)).cuda().float()
                   for i, x in enumerate(sets)], dim=1).contiguous()
    G = torch.randn_like(Q)
    U, V = torch.empty_like(Q), torch.empty_like(Q)
    m.apply_into(Q, U, nrhs, "fp32_tc")
    m.apply_into(G, V, nrhs, "fp32_tc", transpose=True)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            m.apply_into(Q, U, nrhs, "fp32_tc")
            m.apply_into(G, V, nrhs, "fp32_tc", transpose=True)
    Q.mul_(-2.0)
    g.replay()
    torch.cuda.synchronize()
    U2, V2 = torch.empty_like(Q), torch.empty_like(Q)
    m.apply_into(Q, U2, nrhs, "fp32_tc")
    m.apply_into(G, V2, nrhs, "fp32_tc", transpose=True)
    torch.cuda.synchronize()
    assert torch.equal(U, U2) and torch.equal(V, V2)
    m.close()
    b.close()


def test_gmres_with_skeleton_apply():
    """Iterative-solver use: restarted GMRES on (sigma I + A~) x = b with the
    GPU apply as the product, three right-hand sides at once. The solution
    satisfies the system assembled densely from the same apply (to rounding)
    and solves the exact kernel system to about tol * condition. For these
    1200 uniform points the kernel matrix has eigenvalues in [-11.7, 183]
    (computed densely), so sigma = 20 gives a positive definite system with
    condition number 24."""
    from paper_2310_16668_gb300.solve import gmres
    x = W.points_uniform(1200, 3, 41)
    n = x.shape[0]
    fmm = SkelFMM(x, "laplace3d", 1e-9, 16, nrhs_max=16)
    sigma = 20.0
    b = torch.from_numpy(W.charges_normal(n, 3, 42)).cuda()
    sol, info = gmres(fmm, b, sigma=sigma, precision="fp64", restart=40, rtol=1e-11)
    assert info["relres"].max() < 1e-10
    # the same system, assembled densely from the apply: columns of sigma I + A~
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    A = torch.cat([fmm.apply(eye[:, j:j + 16].contiguous(), "fp64") for j in range(0, n, 16)], dim=1)
    M = A + sigma * eye
    assert torch.linalg.vector_norm(M @ sol - b) / torch.linalg.vector_norm(b) < 1e-9
    # against the exact kernel matrix (oracle direct sum) the residual is the
    # compression error: about tol relative to the matrix norm
    sol_np = sol.cpu().numpy()
    Ax = direct.direct_sum("laplace3d", x, sol_np)
    res = np.linalg.norm(Ax + sigma * sol_np - b.cpu().numpy()) / np.linalg.norm(b.cpu().numpy())
    assert res < 1e-6
