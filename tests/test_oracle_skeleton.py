"""Pins for the oracle's proxy surfaces and interpolative decompositions
(Section 2.1, Algorithm 1)."""
import numpy as np
import pytest

from oracle import skeleton as osk
from oracle import tree as otree
from paper_2310_16668_gb300 import workloads as W


@pytest.mark.parametrize("dim,p", [(2, 8), (3, 5)])
def test_proxy_points_on_box_boundary(dim, p):
    c = np.array([0.3, -0.2, 0.7][:dim])
    a = 0.25
    P = osk.proxy_points(c, a, dim, p)
    assert P.shape == ((4 * p, 2) if dim == 2 else (6 * p * p, 3))
    h = 0.5 * 2.95 * a
    off = np.abs(P - c)
    # every point on the boundary of the 2.95a box, none on an edge/corner
    on_face = np.isclose(off, h, rtol=0, atol=1e-14)
    assert np.all(on_face.sum(axis=1) == 1)
    assert np.all(off <= h + 1e-14)
    assert len({tuple(np.round(r, 12)) for r in P}) == P.shape[0]


def test_chebyshev_nodes_first_kind():
    t = osk.chebyshev_nodes(7)
    # zeros of T_7: cos(7 arccos t) = 0
    assert np.allclose(np.cos(7 * np.arccos(t)), 0, atol=1e-14)


@pytest.mark.parametrize("dtype", [np.float64, np.complex128])
def test_id_exact_on_exact_rank(dtype):
    rng = np.random.default_rng(0)
    r = 9
    f = rng.standard_normal((60, r))
    g = rng.standard_normal((r, 40))
    if dtype == np.complex128:
        f = f + 1j * rng.standard_normal((60, r))
        g = g + 1j * rng.standard_normal((r, 40))
    a = f @ g
    piv, k, t = osk.interpolative_decomposition(a, 1e-12)
    assert k == r
    s, rr = piv[:k], piv[k:]
    res = np.linalg.norm(a[:, rr] - a[:, s] @ t) / np.linalg.norm(a)
    assert res < 1e-12
    # T is the unique least-squares solution on the (full column rank) skeleton
    t_ls = np.linalg.lstsq(a[:, s], a[:, rr], rcond=None)[0]
    assert np.allclose(t, t_ls, rtol=0, atol=1e-9 * np.abs(t_ls).max())


@pytest.mark.parametrize("kind,dim", [("laplace2d", 2), ("laplace3d", 3), ("helmholtz3d", 3)])
def test_id_residual_and_rank_monotone(kind, dim):
    x = W.points_uniform(200, dim, 4) * 0.125 + 0.4
    c = np.full(dim, 0.4 + 0.0625)
    P = osk.proxy_points(c, 0.125, dim, osk.DEFAULT_P[dim])
    m = osk.proxy_matrix(kind, P, x, 25.0)
    ks = []
    for tol in (1e-2, 1e-4, 1e-6, 1e-8):
        piv, k, t = osk.interpolative_decomposition(m, tol)
        res = np.linalg.norm(m[:, piv[k:]] - m[:, piv[:k]] @ t, 2) / np.linalg.norm(m, 2)
        assert res <= 30 * tol
        ks.append(k)
    assert ks == sorted(ks) and ks[0] < ks[-1]


def test_far_field_interpolation_beyond_proxy():
    """The proxy ID of a box interpolates the kernel for sources anywhere
    outside the proxy box (the reason proxies replace the far field)."""
    dim = 3
    box_c, a = np.array([0.5, 0.5, 0.5]), 0.25
    x = box_c + (W.points_uniform(150, dim, 9) - 0.5) * a
    m = osk.proxy_matrix("laplace3d", osk.proxy_points(box_c, a, dim, 12), x, 0.0)
    tol = 1e-7
    piv, k, t = osk.interpolative_decomposition(m, tol)
    far = box_c + (W.points_uniform(3000, dim, 10) - 0.5) * 6 * a
    far = far[np.max(np.abs(far - box_c), axis=1) > 0.5 * 3 * a]
    from oracle.kernels import kernel_matrix
    g = kernel_matrix("laplace3d", far, x)
    err = np.linalg.norm(g[:, piv[k:]] - g[:, piv[:k]] @ t) / np.linalg.norm(g)
    assert err < 100 * tol


def test_tree_index_sets_are_child_skeletons():
    t = otree.Tree(W.points_uniform(2500, 3, 1), 20)
    sk = osk.Skeletons(t, "laplace3d", 1e-5)
    for b in range(1, t.n_boxes):
        if not t.is_leaf[b]:
            cat = np.concatenate([sk.skel(c) for c in t.children[b]])
            assert np.array_equal(sk.idx[b], cat)
        else:
            assert np.array_equal(np.sort(sk.idx[b]), t.points[b])
        assert sorted(sk.piv[b].tolist()) == list(range(len(sk.idx[b])))
        assert sk.T[b].shape == (sk.k[b], len(sk.idx[b]) - sk.k[b])
