"""C-ABI checks that need no GPU: the library loads and exports every symbol
of include/skel.h, argument validation, and the host build (tree, neighbor
lists, interpolative decompositions) against the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import apply as oap
from oracle import direct
from oracle import plan as oplan
from oracle import skeleton as osk
from oracle import tree as otree
from paper_2310_16668_gb300 import SkelFMM, _lib
from paper_2310_16668_gb300 import workloads as W
from tests._util import clustered, relerr, skeletons_from_plan

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "skel.h")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_16668_gb300 import build
    build.build()


def test_library_exports_every_header_symbol():
    decl = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(skel_\w+)\s*\(", open(HEADER).read(), re.M))
    assert decl == set(_lib.SYMBOLS)
    lib = _lib.load()
    for name in decl:
        assert hasattr(lib, name), name


CASES = [("laplace2d", 2, 3000, 12, 1e-8), ("laplace3d", 3, 3000, 16, 1e-6), ("helmholtz3d", 3, 2500, 16, 1e-6),
         ("helmholtz2d", 2, 2500, 16, 1e-8)]


@pytest.mark.parametrize("kind,dim,n,b,tol", CASES)
def test_host_build_matches_oracle(kind, dim, n, b, tol):
    x = clustered(n, dim, 1)
    f = SkelFMM(x, kind, tol, b, kappa=25.0, host_only=True)
    pl = f.export_plan()
    t = otree.Tree(x, b)
    # tree: bit-exact
    assert t.n_boxes == pl["level"].shape[0]
    assert np.array_equal(t.level, pl["level"])
    assert np.array_equal(np.array(t.coord), pl["coord"])
    assert np.array_equal(t.parent, pl["parent"])
    assert np.array_equal(t.is_leaf.astype(np.int8), pl["is_leaf"])
    assert np.allclose(pl["center"], t.center, rtol=0, atol=0) and pl["side"] == t.side
    for leaf in t.leaves():
        got = pl["idx"][pl["idx_ptr"][leaf]:pl["idx_ptr"][leaf + 1]]
        assert np.array_equal(got, t.points[leaf])
    # neighbor lists: bit-exact
    for which, lists in ((0, t.colleagues), (1, t.coarse), (2, t.fine)):
        ptr, lst = f.neighbors(which)
        for bx in range(t.n_boxes):
            assert list(lst[ptr[bx]:ptr[bx + 1]]) == lists[bx]
    # IDs: library T on the oracle's own proxy matrix, and ranks vs the oracle
    assert f.info()["n_proxy"] == len(osk.proxy_points(t.box_center(0), t.box_side(0), dim, osk.DEFAULT_P[dim]))
    sk = osk.Skeletons(t, kind, tol, kappa=25.0)
    ip, tp = pl["idx_ptr"], pl["T_ptr"]
    for bx in range(t.n_boxes):
        if t.level[bx] < 2:
            continue
        I = pl["idx"][ip[bx]:ip[bx + 1]]
        piv = pl["piv"][ip[bx]:ip[bx + 1]]
        k = int(pl["k"][bx])
        T = np.asarray(pl["T"][tp[bx]:tp[bx + 1]]).reshape((k, len(I) - k), order="F")
        m = osk.proxy_matrix(kind, osk.proxy_points(t.box_center(bx), t.box_side(bx), dim,
                                                    osk.DEFAULT_P[dim]), x[I], 25.0)
        res = np.linalg.norm(m[:, piv[k:]] - m[:, piv[:k]] @ T, 2) if k < len(I) else 0.0
        assert res <= 30 * tol * np.linalg.norm(m, 2)
        assert abs(k - int(sk.k[bx])) <= 1
    # the library's operators drive the oracle's Algorithm 2 to the direct sum
    q = (W.charges_complex if kind in ("helmholtz3d", "helmholtz2d") else W.charges_normal)(x.shape[0], 1, 2)[:, 0]
    u = oap.skeleton_apply(skeletons_from_plan(t, kind, pl, kappa=25.0), q)
    assert relerr(u, direct.direct_sum(kind, x, q, kappa=25.0)) < 10 * tol


def test_export_import_roundtrip_host_only():
    x = clustered(2000, 3, 3)
    sk = osk.Skeletons(otree.Tree(x, 16), "laplace3d", 1e-5)
    plan = oplan.to_exchange(sk)
    f = SkelFMM.from_plan(x, "laplace3d", plan, host_only=True)
    back = f.export_plan()
    for key in ("level", "coord", "parent", "is_leaf", "idx_ptr", "idx", "piv", "k", "T_ptr"):
        assert np.array_equal(np.asarray(back[key]).ravel(), np.asarray(plan[key]).ravel()), key
    assert np.array_equal(back["T"], plan["T"])


def _expect(code, fn, *a, **kw):
    with pytest.raises(_lib.SkelError) as e:
        fn(*a, **kw)
    assert e.value.code == code, str(e.value)


def test_import_rejects_inconsistent_plans():
    x = clustered(1500, 3, 4)
    sk = osk.Skeletons(otree.Tree(x, 16), "laplace3d", 1e-5)
    good = oplan.to_exchange(sk)

    def bad(**changes):
        p = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in good.items()}
        for k, f in changes.items():
            f(p[k])
        _expect(-1, SkelFMM.from_plan, x, "laplace3d", p, host_only=True)

    nb = good["level"].shape[0]
    leaf = int(np.nonzero(good["is_leaf"])[0][-1])
    tree_box = int(np.nonzero((good["is_leaf"] == 0) & (good["level"] >= 2))[0][0])

    def swap_idx(a):
        lo = good["idx_ptr"][tree_box]
        a[lo], a[lo + 1] = a[lo + 1], a[lo]

    bad(idx=swap_idx)                                              # not the children's skeletons
    bad(piv=lambda a: a.__setitem__(good["idx_ptr"][leaf], a[good["idx_ptr"][leaf] + 1]))  # not a permutation
    bad(parent=lambda a: a.__setitem__(nb - 1, 0))                  # wrong parent
    bad(is_leaf=lambda a: a.__setitem__(tree_box, 1))               # leaf with children
    bad(k=lambda a: a.__setitem__(leaf, 0))                         # k out of range
    bad(coord=lambda a: a.__setitem__((leaf, 0), a[leaf, 0] ^ 1))   # box moved away from its points


def lib_autotune_null():
    return _lib.load().skel_autotune(None, 4, 1, None, None)


def test_argument_errors():
    x = W.points_uniform(300, 3, 0)
    _expect(-1, SkelFMM, x, "laplace3d", 0.0, 16, host_only=True)        # tol
    _expect(-1, SkelFMM, x, "laplace3d", 1e-6, 0, host_only=True)        # leaf size
    _expect(-1, SkelFMM, x[:, :2], "laplace3d", 1e-6, 16, host_only=True)  # dim vs kernel
    bad = x.copy()
    bad[5, 1] = np.nan
    _expect(-5, SkelFMM, bad, "laplace3d", 1e-6, 16, host_only=True)     # non-finite
    _expect(-1, SkelFMM, x, "laplace3d", 1e-6, 16, host_only=True, device_build=True)  # needs a device
    f = SkelFMM(x, "laplace3d", 1e-6, 16, host_only=True)
    _expect(-6, f.apply, np.zeros(300))                                   # host-only plan
    _expect(-6, f.autotune, 4)                                            # nothing to tune on the host
    assert lib_autotune_null() == -1
    lib = _lib.load()
    assert lib.skel_apply(None, None, None, 1, 0, None) == -1
    lib.skel_free(None)                                                   # NULL is a no-op
    assert lib.skel_info(None, None) == -1
    # failure-detection test hooks: argument checks (no device needed)
    assert lib.skel_test_fail_alloc(-1) == -1
    assert lib.skel_test_fail_alloc(0) == 0                               # off
    assert lib.skel_test_withhold_tile(None, 5.0) == -1
    assert lib.skel_test_withhold_tile(f._h, 5.0) == -6                   # host-only plan
    assert lib.skel_test_set_updown(None, 0) == -1
    assert lib.skel_test_set_updown(f._h, 0) == -6                       # host-only plan


def test_single_leaf_root_plan():
    x = W.points_uniform(40, 3, 2)
    f = SkelFMM(x, "laplace3d", 1e-6, 64, host_only=True)
    info = f.info()
    assert info["n_levels"] == 0 and info["n_boxes"] == 1
    assert info["pairs_direct"] == 40 * 40 and info["pairs_far"] == 0


@pytest.mark.parametrize("threads", [2, 64])
def test_build_batch_equals_single_builds(threads):
    # threads = 2: sets built in parallel, one thread each; 64: one after
    # the other with all threads. Either way each plan is the single build's.
    from paper_2310_16668_gb300 import SkelBatch
    sets = [W.points_curve(n, 100 + i) for i, n in enumerate((300, 1200, 50, 2000, 1))]
    b = SkelBatch(sets, "laplace2d", 1e-7, 16, num_threads=threads, host_only=True)
    assert b.sizes == [len(x) for x in sets]
    for x, f in zip(sets, b.plans):
        g = SkelFMM(x, "laplace2d", 1e-7, 16, host_only=True)
        pa, pb = f.export_plan(), g.export_plan()
        assert pa.keys() == pb.keys()
        for key in pa:
            assert np.array_equal(np.asarray(pa[key]), np.asarray(pb[key])), key


def test_merged_layout_sums_the_sets():
    """skel_merge (host part): the merged layout holds exactly the sets' boxes,
    entries, operators and translation work; plan export is refused."""
    from paper_2310_16668_gb300 import SkelBatch
    sets = [W.points_curve(n, 900 + i) for i, n in enumerate((700, 1500, 2600, 1100))]
    b = SkelBatch(sets, "laplace2d", 1e-7, 16, nrhs_max=4, host_only=True)
    m = b.merged(host_only=True)
    mi, infos = m.info(), [f.info() for f in b.plans]
    for k in ("n_points", "n_boxes", "n_leaves", "n_index", "n_T", "pairs_direct", "pairs_far", "pairs_tc",
              "n_tc_items", "n_tc_tiles", "n_mix_items", "n_work_items", "n_colleague", "n_coarse", "n_fine"):
        assert mi[k] == sum(i[k] for i in infos), k
    assert mi["k_max"] == max(i["k_max"] for i in infos)
    assert mi["n_levels"] == max(i["n_levels"] for i in infos)
    _expect(-6, m.export_plan)
    _expect(-6, m.apply, np.zeros(mi["n_points"]))
    b3 = SkelBatch([W.points_uniform(500, 3, 1)], "laplace3d", 1e-6, 16, host_only=True)
    lib = _lib.load()
    hs = (ctypes.c_void_p * 2)(b.plans[0]._h.value, b3.plans[0]._h.value)
    out = ctypes.c_void_p()
    assert lib.skel_merge(hs, 2, None, ctypes.byref(out)) == -1          # kernels differ
    assert out.value is None


def test_build_batch_errors_name_the_set():
    from paper_2310_16668_gb300 import SkelBatch
    from paper_2310_16668_gb300._lib import SkelError
    sets = [W.points_uniform(100, 2, i) for i in range(4)]
    sets[2] = sets[2].copy()
    sets[2][7, 0] = np.inf
    with pytest.raises(SkelError) as e:
        SkelBatch(sets, "laplace2d", 1e-7, 16, host_only=True)
    assert e.value.code == -5
    with pytest.raises(SkelError) as e:
        SkelBatch([W.points_uniform(100, 2, 0)] * 2, "laplace2d", 2.0, 16, host_only=True)   # tol
    assert e.value.code == -1
    with pytest.raises(SkelError) as e:                                                       # device build, no device
        SkelBatch([W.points_uniform(100, 2, 0)], "laplace2d", 1e-7, 16, host_only=True, device_build=True)
    assert e.value.code == -1
    lib = _lib.load()
    assert lib.skel_build_batch(0, None, None, 2, _lib.SkelKernel(0, 0.0), 1e-7, 16, None, None) == -1
