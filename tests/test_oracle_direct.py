"""Pins for the oracle's kernels and direct sum (Section 1, Eq. (1)-(2), (5)).

The direct sum is checked against (a) closed forms on small symmetric point
configurations, (b) a pure-Python double loop over pairs that uses only
``math`` scalars (independent of ``kernels.kernel_matrix``), and (c) the C
loop against the numpy blocks.
"""
import math

import numpy as np
import pytest

from oracle import direct, kernels
from paper_2310_16668_gb300 import workloads as W


def test_kernel_closed_forms():
    assert kernels.kernel_scalar("laplace3d", 1.0) == pytest.approx(1.0 / (4 * math.pi), rel=1e-15)
    assert kernels.kernel_scalar("laplace3d", 0.5) == pytest.approx(1.0 / (2 * math.pi), rel=1e-15)
    assert kernels.kernel_scalar("laplace2d", 1.0) == 0.0
    assert kernels.kernel_scalar("laplace2d", math.e) == pytest.approx(-1.0 / (2 * math.pi), rel=1e-15)
    g = kernels.kernel_scalar("helmholtz3d", 1.0, kappa=math.pi)
    assert g.real == pytest.approx(-1.0 / (4 * math.pi), rel=1e-14)
    assert abs(g.imag) < 1e-16
    g = kernels.kernel_scalar("helmholtz3d", 0.5, kappa=math.pi)   # e^{i pi/2} / (2 pi)
    assert abs(g.real) < 1e-16 and g.imag == pytest.approx(1.0 / (2 * math.pi), rel=1e-14)


def test_helmholtz2d_published_values_and_laplace_limit():
    """2D Helmholtz G = (i/4) H_0^(1)(kappa r) = (-Y_0 + i J_0) / 4 at
    kappa r = 1, with J_0(1) and Y_0(1) from Abramowitz and Stegun, Table 9.1;
    and for kappa -> 0, G minus the 2D Laplace kernel -log(r)/(2 pi) tends to
    the r-independent constant -(log(kappa / 2) + Euler's gamma)/(2 pi) + i/4
    (the small-argument form of Y_0, A&S 9.1.13)."""
    j0_1, y0_1 = 0.765197686557966551, 0.088256964215676958
    g = kernels.kernel_scalar("helmholtz2d", 1.0, kappa=1.0)
    assert g.real == pytest.approx(-y0_1 / 4, rel=1e-13)
    assert g.imag == pytest.approx(j0_1 / 4, rel=1e-13)
    g2 = kernels.kernel_scalar("helmholtz2d", 0.5, kappa=2.0)        # same kappa r
    assert abs(g2 - g) < 1e-15
    kappa, gamma = 1e-7, 0.5772156649015329
    limit = complex(-(math.log(kappa / 2) + gamma) / (2 * math.pi), 0.25)
    for r in (0.01, 0.3, 2.0):
        d = kernels.kernel_scalar("helmholtz2d", r, kappa=kappa) - kernels.kernel_scalar("laplace2d", r)
        assert abs(d - limit) < 1e-9


@pytest.mark.parametrize("kind", ["laplace2d", "laplace3d", "helmholtz3d", "helmholtz2d", "poly2"])
def test_zero_diagonal_and_coincident(kind):
    dim = 2 if kind in ("laplace2d", "helmholtz2d") else 3
    x = W.points_uniform(5, dim, 0)
    x = np.vstack([x, x[2:3]])       # a duplicated point
    g = kernels.kernel_matrix(kind, x, x, kappa=3.0)
    assert np.all(np.diag(g) == 0)
    assert g[2, 5] == 0 and g[5, 2] == 0
    assert np.allclose(g, g.T, rtol=1e-15, atol=0)


def test_cube_vertices_closed_form():
    # unit charges on the 8 vertices of the unit cube: at a vertex the other
    # vertices sit at distance 1 (3 of them), sqrt 2 (3) and sqrt 3 (1)
    x = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float)
    q = np.ones(8)
    expect = (3.0 + 3.0 / math.sqrt(2) + 1.0 / math.sqrt(3)) / (4 * math.pi)
    for u in (direct.direct_sum("laplace3d", x, q), direct.direct_sum_numpy("laplace3d", x, q)):
        assert np.allclose(u, expect, rtol=1e-14, atol=0)


def test_square_vertices_closed_form():
    # unit square, unit charges: -(log 1 + log 1 + log sqrt 2) / (2 pi) = -log 2 / (4 pi)
    x = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=float)
    u = direct.direct_sum("laplace2d", x, np.ones(4))
    assert np.allclose(u, -math.log(2) / (4 * math.pi), rtol=1e-14, atol=0)


def test_two_point_helmholtz():
    kappa, r = 7.0, 0.3
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    q = np.array([0.0 + 0j, 2.0 - 1.0j])
    u = direct.direct_sum("helmholtz3d", x, q, kappa=kappa)
    expect = np.exp(1j * kappa * r) / (4 * math.pi * r) * q[1]
    assert abs(u[0] - expect) < 1e-14 * abs(expect) and u[1] == pytest.approx(
        np.exp(1j * kappa * r) / (4 * math.pi * r) * q[0])


def _python_pairs(kind, x, q, kappa):
    n = x.shape[0]
    out = []
    for i in range(n):
        acc = 0j
        for j in range(n):
            d = math.sqrt(sum((x[i, k] - x[j, k]) ** 2 for k in range(x.shape[1])))
            if d == 0.0:
                continue
            if kind == "laplace2d":
                g = -math.log(d) / (2 * math.pi)
            elif kind == "laplace3d":
                g = 1.0 / (4 * math.pi * d)
            else:
                g = complex(math.cos(kappa * d), math.sin(kappa * d)) / (4 * math.pi * d)
            acc += g * q[j]
        out.append(acc)
    return np.array(out)


@pytest.mark.parametrize("kind,dim", [("laplace2d", 2), ("laplace3d", 3), ("helmholtz3d", 3)])
def test_direct_vs_python_pairs(kind, dim):
    x = W.points_uniform(40, dim, 7)
    q = W.charges_complex(40, 1, 8)[:, 0] if kind == "helmholtz3d" else W.charges_normal(40, 1, 8)[:, 0]
    ref = _python_pairs(kind, x, q, 25.0)
    if kind != "helmholtz3d":
        ref = ref.real
    for u in (direct.direct_sum(kind, x, q, kappa=25.0), direct.direct_sum_numpy(kind, x, q, kappa=25.0)):
        assert np.allclose(u, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("kind,dim", [("laplace2d", 2), ("laplace3d", 3), ("helmholtz3d", 3), ("helmholtz2d", 2)])
def test_c_vs_numpy_multi_rhs_and_targets(kind, dim):
    n = 700
    x = W.points_uniform(n, dim, 11)
    q = W.charges_complex(n, 3, 12) if kind == "helmholtz3d" else W.charges_normal(n, 3, 12)
    tg = W.sample_targets(n, 50, 13)
    a = direct.direct_sum(kind, x, q, targets=tg, kappa=25.0)
    b = direct.direct_sum_numpy(kind, x, q, targets=tg, kappa=25.0)
    assert a.shape == (50, 3)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(b).max())


def test_translation_invariance_and_symmetry():
    x = W.points_uniform(300, 3, 21)
    q = W.charges_normal(300, 1, 22)[:, 0]
    p = W.charges_normal(300, 1, 23)[:, 0]
    u = direct.direct_sum("laplace3d", x, q)
    v = direct.direct_sum("laplace3d", x + np.array([5.0, -3.0, 2.0]), q)
    assert np.allclose(u, v, rtol=1e-12, atol=1e-12 * np.abs(u).max())
    lhs = np.dot(direct.direct_sum("laplace3d", x, q), p)
    rhs = np.dot(q, direct.direct_sum("laplace3d", x, p))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
