"""Algorithm 1 on the GPU (``device_build``) against the oracle and the host build.

The device build runs the same steps as the host build (proxy matrix, pivoted
QR stopped at |R_jj| <= tol |R_00|, T = R_11^{-1} R_12) in FP64 on the GPU, so
its IDs are checked the way the host build's are: T reproduces the oracle's
own proxy matrix to the ID tolerance, the ranks are within one of the
oracle's, and the operators drive the oracle's Algorithm 2 to the direct sum.
"""
import numpy as np
import pytest
import torch

from oracle import apply as oap
from oracle import direct
from oracle import skeleton as osk
from oracle import tree as otree
from paper_2310_16668_gb300 import SkelFMM
from paper_2310_16668_gb300 import workloads as W
from tests._util import clustered, relerr, skeletons_from_plan

pytestmark = pytest.mark.gpu
KAPPA = 25.0


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_16668_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _charges(kind, n, seed):
    f = W.charges_complex if kind in ("helmholtz3d", "helmholtz2d") else W.charges_normal
    return f(n, 1, seed)[:, 0]


CASES = [("laplace2d", 2, 3000, 12, 1e-8), ("laplace3d", 3, 3000, 16, 1e-6), ("helmholtz3d", 3, 2500, 16, 1e-6),
         ("helmholtz2d", 2, 2500, 16, 1e-8), ("laplace3d", 3, 4000, 24, 1e-10)]


@pytest.mark.parametrize("kind,dim,n,b,tol", CASES)
def test_device_build_matches_oracle(kind, dim, n, b, tol):
    x = clustered(n, dim, 1)
    f = SkelFMM(x, kind, tol, b, kappa=KAPPA, device_build=True)
    info = f.info()
    assert info["skel_on_device"] == 1 and info["t_id_kernels"] > 0 and info["id_gflop"] > 0
    pl = f.export_plan()
    t = otree.Tree(x, b)
    sk = osk.Skeletons(t, kind, tol, kappa=KAPPA)
    ip, tp = pl["idx_ptr"], pl["T_ptr"]
    for bx in range(t.n_boxes):
        I = pl["idx"][ip[bx]:ip[bx + 1]]
        piv = pl["piv"][ip[bx]:ip[bx + 1]]
        k = int(pl["k"][bx])
        assert sorted(piv) == list(range(len(I)))
        if t.level[bx] < 2:
            assert k == len(I)
            continue
        T = np.asarray(pl["T"][tp[bx]:tp[bx + 1]]).reshape((k, len(I) - k), order="F")
        m = osk.proxy_matrix(kind, osk.proxy_points(t.box_center(bx), t.box_side(bx), dim,
                                                    osk.DEFAULT_P[dim]), x[I], KAPPA)
        res = np.linalg.norm(m[:, piv[k:]] - m[:, piv[:k]] @ T, 2) if k < len(I) else 0.0
        assert res <= 30 * tol * np.linalg.norm(m, 2)
        assert abs(k - int(sk.k[bx])) <= 1
    q = _charges(kind, x.shape[0], 2)
    ref = direct.direct_sum(kind, x, q, kappa=KAPPA)
    # the device-built operators drive the oracle's Algorithm 2 and the GPU apply
    u = oap.skeleton_apply(skeletons_from_plan(t, kind, pl, kappa=KAPPA), q)
    assert relerr(u, ref) < 10 * tol
    ug = f.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    assert relerr(ug, ref) < 10 * tol
    assert relerr(ug, u) < 1e-12


@pytest.mark.parametrize("kind,dim,tol", [("laplace3d", 3, 1e-6), ("helmholtz2d", 2, 1e-8)])
def test_device_build_agrees_with_host_build(kind, dim, tol):
    x = clustered(6000, dim, 3)
    fd = SkelFMM(x, kind, tol, 24, kappa=KAPPA, device_build=True)
    fh = SkelFMM(x, kind, tol, 24, kappa=KAPPA)
    pd, ph = fd.export_plan(), fh.export_plan()
    kd, kh = np.asarray(pd["k"]), np.asarray(ph["k"])
    assert np.abs(kd - kh).max() <= 2
    assert np.mean(kd == kh) > 0.9
    q = _charges(kind, x.shape[0], 4)
    qt = torch.from_numpy(q).cuda()
    ud = fd.apply(qt, "fp64").cpu().numpy()
    uh = fh.apply(qt, "fp64").cpu().numpy()
    assert relerr(ud, uh) < 10 * tol


def test_device_build_degenerate_inputs():
    # coincident points (equal columns: exact pivot-norm ties), a single leaf,
    # and two points
    x = W.points_uniform(2000, 3, 6)
    x[100:110] = x[5]
    q = W.charges_normal(2000, 1, 7)[:, 0]
    f = SkelFMM(x, "laplace3d", 1e-6, 16, device_build=True)
    u = f.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    assert relerr(u, direct.direct_sum("laplace3d", x, q)) < 1e-5
    for n in (2, 40):
        x = W.points_uniform(n, 3, 2)
        q = W.charges_normal(n, 1, 3)[:, 0]
        f = SkelFMM(x, "laplace3d", 1e-6, 64, device_build=True)
        u = f.apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
        assert relerr(u, direct.direct_sum("laplace3d", x, q)) < 1e-13


@pytest.mark.slow
def test_full_size_device_build():
    wl = W.LAPLACE3D_1M
    x = wl.make_points()
    qall = wl.make_charges(32)
    f = SkelFMM(x, wl.kernel, wl.tol, wl.leaf, nrhs_max=32, device_build=True)
    tg = wl.make_sample()
    ref = direct.direct_sum(wl.kernel, x, np.ascontiguousarray(qall[:, 0]), targets=tg)
    utc = f.apply(torch.from_numpy(qall).cuda().float(), "fp32_tc").cpu().numpy()
    info = f.info()
    e = relerr(utc[tg, 0], ref)
    print(f"device build: t_skel {info['t_skel']:.2f} s (kernels {info['t_id_kernels']:.2f} s, "
          f"{info['id_gflop']:.0f} GFLOP), k_max {info['k_max']}, n_T {info['n_T']}, relerr fp32_tc {e:.3e}")
    assert e < 10 * wl.tol
