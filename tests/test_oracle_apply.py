"""Pins for the oracle's Algorithm 2 apply.

* Exactly low-rank kernel (poly2): every ID is exact, so the skeleton apply
  must equal the direct sum to rounding on uniform and adaptive trees (with
  coarse and fine neighbors). A dropped or doubled term, a wrong sign, a wrong
  slot or T in place of T^* all break this.
* Matrix form: on a two-level uniform tree the operator assembled column by
  column equals the sparse factorisation of Section 2.3,
  A^near - E A_SS^near F + E A_SS F (Eq. (e:mod_near)), built from the IDs.
* Laplace / Helmholtz accuracy: error vs the direct sum below 10 tol, and
  decreasing as tol tightens while ranks grow (Section 5 tables).
* Symmetry / transpose, linearity, the single-leaf root and the keep-all ID.
"""
import numpy as np
import pytest

from oracle import apply as oap
from oracle import direct, kernels
from oracle import skeleton as osk
from oracle import tree as otree
from paper_2310_16668_gb300 import workloads as W


def _clustered(n, dim, seed, frac=4, sigma=0.01, c=0.41):
    x = W.points_uniform(n, dim, seed)
    rng = np.random.default_rng(seed + 1)
    return np.vstack([x, c + sigma * rng.standard_normal((n // frac, dim))])


def _relerr(u, ref):
    return np.abs(u - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("dim,n,b,adaptive", [(2, 1500, 8, False), (2, 1500, 6, True),
                                               (3, 2500, 5, False), (3, 2000, 10, True)])
def test_poly_kernel_exact(dim, n, b, adaptive):
    # cluster width 0.03: deep enough for coarse/fine neighbors, while the
    # quadratic basis stays well resolved at tol 1e-13 in the smallest boxes
    x = _clustered(n, dim, 2, sigma=0.03) if adaptive else W.points_uniform(n, dim, 2)
    q = W.charges_normal(x.shape[0], 2, 3)
    t = otree.Tree(x, b)
    assert t.n_levels >= 4
    if adaptive:
        assert sum(map(len, t.coarse)) > 0 and sum(map(len, t.fine)) > 0
    sk = osk.Skeletons(t, "poly2", 1e-13)
    assert sk.k_max() == (6 if dim == 2 else 10)
    u = oap.skeleton_apply(sk, q)
    ref = direct.direct_sum_numpy("poly2", x, q)
    assert _relerr(u, ref) < 1e-11


def test_matrix_form_two_levels():
    # jittered 4x4 grid of 10-point clusters: a uniform tree with leaves at level 2
    rng = np.random.default_rng(7)
    cells = [(i, j) for i in range(4) for j in range(4)]
    x = np.vstack([(np.array(c) + 0.2 + 0.6 * rng.random((10, 2))) / 4 for c in cells])
    t = otree.Tree(x, 12)
    assert t.n_levels == 2 and all(t.level[l] == 2 for l in t.leaves())
    sk = osk.Skeletons(t, "laplace2d", 1e-4)
    n = x.shape[0]
    # operator of Algorithm 2, column by column
    a_alg = np.column_stack([oap.skeleton_apply(sk, e) for e in np.eye(n)])
    # sparse factorisation of Section 2.3 at the leaf level; level 1 is exact
    a = kernels.kernel_matrix("laplace2d", x, x)
    leaves = t.boxes_at[2]
    near = np.zeros((n, n))
    for b in leaves:
        for c in t.colleagues[b]:
            near[np.ix_(sk.idx[b], sk.idx[c])] = a[np.ix_(sk.idx[b], sk.idx[c])]
    s_all = np.concatenate([sk.skel(b) for b in leaves])
    pos = {int(p): i for i, p in enumerate(s_all)}
    F = np.zeros((len(s_all), n))
    for b in leaves:
        S = sk.piv[b][: sk.k[b]]
        R = sk.piv[b][sk.k[b]:]
        rows = [pos[int(p)] for p in sk.idx[b][S]]
        F[np.ix_(rows, sk.idx[b][S])] = np.eye(len(S))
        F[np.ix_(rows, sk.idx[b][R])] = sk.T[b]
    E = F.T
    ass = a[np.ix_(s_all, s_all)]
    ass_near = np.zeros_like(ass)
    for b in leaves:
        rb = [pos[int(p)] for p in sk.skel(b)]
        for c in t.colleagues[b]:
            rc = [pos[int(p)] for p in sk.skel(c)]
            ass_near[np.ix_(rb, rc)] = ass[np.ix_(rb, rc)]
    a_mat = near - E @ ass_near @ F + E @ ass @ F
    assert np.abs(a_alg - a_mat).max() < 1e-12 * np.abs(a_mat).max()
    # and the factorisation approximates A
    assert np.abs(a_mat - a).max() < 1e-2 * np.abs(a).max()


@pytest.mark.parametrize("kind,dim,b", [("laplace2d", 2, 16), ("laplace3d", 3, 24)])
def test_laplace_accuracy_and_decay(kind, dim, b):
    x = _clustered(3000, dim, 11)
    q = W.charges_normal(x.shape[0], 1, 12)[:, 0]
    ref = direct.direct_sum(kind, x, q)
    t = otree.Tree(x, b)
    errs, kmax = [], []
    for tol in (1e-3, 1e-5, 1e-7):
        sk = osk.Skeletons(t, kind, tol)
        e = _relerr(oap.skeleton_apply(sk, q), ref)
        assert e <= 10 * tol
        errs.append(e)
        kmax.append(sk.k_max())
    assert errs[0] > errs[1] > errs[2]
    assert kmax[0] < kmax[1] < kmax[2]


def test_helmholtz_accuracy_and_transpose():
    x = _clustered(2000, 3, 13)
    n = x.shape[0]
    q = W.charges_complex(n, 1, 14)[:, 0]
    p = W.charges_complex(n, 1, 15)[:, 0]
    t = otree.Tree(x, 24)
    sk = osk.Skeletons(t, "helmholtz3d", 1e-6, kappa=25.0)
    u = oap.skeleton_apply(sk, q)
    ref = direct.direct_sum("helmholtz3d", x, q, kappa=25.0)
    assert _relerr(u, ref) < 1e-5
    # bilinear transpose identity <A q, p> = <q, A^T p>
    lhs = np.sum(u * p)
    rhs = np.sum(q * oap.skeleton_apply(sk, p, transpose=True))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the transpose differs from the plain apply for a complex ID
    assert np.abs(oap.skeleton_apply(sk, p, transpose=True) - oap.skeleton_apply(sk, p)).max() > 0


def test_laplace_symmetry_and_linearity():
    x = _clustered(2500, 3, 17)
    n = x.shape[0]
    q = W.charges_normal(n, 1, 18)[:, 0]
    p = W.charges_normal(n, 1, 19)[:, 0]
    sk = osk.Skeletons(otree.Tree(x, 16), "laplace3d", 1e-4)
    uq = oap.skeleton_apply(sk, q)
    up = oap.skeleton_apply(sk, p)
    assert abs(np.dot(uq, p) - np.dot(q, up)) < 1e-12 * abs(np.dot(uq, p))
    both = oap.skeleton_apply(sk, np.column_stack([q, 2.5 * q - p]))
    assert np.allclose(both[:, 0], uq, rtol=0, atol=1e-13 * np.abs(uq).max())
    assert np.allclose(both[:, 1], 2.5 * uq - up, rtol=0, atol=1e-12 * np.abs(uq).max())


def test_single_leaf_root_is_direct():
    x = W.points_uniform(50, 3, 1)
    q = W.charges_normal(50, 1, 2)[:, 0]
    sk = osk.Skeletons(otree.Tree(x, 64), "laplace3d", 1e-6)
    assert _relerr(oap.skeleton_apply(sk, q), direct.direct_sum("laplace3d", x, q)) < 1e-14


@pytest.mark.parametrize("kind,dim", [("laplace3d", 3), ("laplace2d", 2), ("helmholtz2d", 2)])
def test_keep_all_is_direct(kind, dim):
    x = _clustered(900, dim, 21)
    q = W.charges_normal(x.shape[0], 1, 22)[:, 0]
    if kind == "helmholtz2d":
        q = q + 0.5j * W.charges_normal(x.shape[0], 1, 23)[:, 0]
    sk = osk.Skeletons(otree.Tree(x, 6), kind, 1e-6, keep_all=True, kappa=25.0)
    ref = direct.direct_sum(kind, x, q, kappa=25.0)
    assert _relerr(oap.skeleton_apply(sk, q), ref) < 1e-13


def test_helmholtz2d_accuracy_and_transpose():
    """2D Helmholtz (kappa = 25): the skeleton apply reaches the direct sum
    within 10 tol, and <A~ q, p> = <q, A~^T p> under the bilinear form."""
    x = _clustered(1500, 2, 24)
    n = x.shape[0]
    q = W.charges_complex(n, 1, 25)[:, 0]
    p = W.charges_complex(n, 1, 26)[:, 0]
    sk = osk.Skeletons(otree.Tree(x, 16), "helmholtz2d", 1e-8, kappa=25.0)
    assert _relerr(oap.skeleton_apply(sk, q), direct.direct_sum("helmholtz2d", x, q, kappa=25.0)) < 1e-7
    lhs = np.sum(oap.skeleton_apply(sk, q) * p)
    rhs = np.sum(q * oap.skeleton_apply(sk, p, transpose=True))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_proxy_convergence():
    """Doubling the proxy density does not change the error by more than 2x
    (the proxy surface already resolves the far field)."""
    x = W.points_uniform(3000, 3, 31)
    q = W.charges_normal(3000, 1, 32)[:, 0]
    ref = direct.direct_sum("laplace3d", x, q)
    t = otree.Tree(x, 24)
    e = [_relerr(oap.skeleton_apply(osk.Skeletons(t, "laplace3d", 1e-6, proxy_p=p), q), ref)
         for p in (osk.DEFAULT_P[3], 2 * osk.DEFAULT_P[3])]
    assert e[0] < 2 * e[1] and e[0] < 1e-5
