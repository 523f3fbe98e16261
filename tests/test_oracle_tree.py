"""Pins for the oracle tree (Section 3.1): a hand-derived golden tree, the
structural invariants of the paper's tree, and neighbor lists checked against
a floating-point geometric test that shares nothing with the integer one."""
import os

import numpy as np
import pytest

from oracle import tree as otree
from paper_2310_16668_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tree_2d_b1.txt")


def _clustered(n, dim, seed):
    x = W.points_uniform(n, dim, seed)
    rng = np.random.default_rng(seed + 1)
    c = 0.37 + 0.004 * rng.standard_normal((n // 3, dim))
    return np.vstack([x, c])


def test_golden_tree():
    x = np.array([[0, 0], [1, 1], [0.30, 0.30], [0.31, 0.31]], dtype=float)
    t = otree.Tree(x, 1)
    boxes, rel = set(), set()
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "box":
            pts = () if f[5] == "-" else tuple(int(v) for v in f[5].split(","))
            boxes.add((int(f[1]), (int(f[2]), int(f[3])), bool(int(f[4])), pts))
        else:
            rel.add((f[0], (int(f[1]), (int(f[2]), int(f[3]))), (int(f[4]), (int(f[5]), int(f[6])))))
    got = set()
    for b in range(t.n_boxes):
        pts = tuple(int(v) for v in t.points[b]) if t.is_leaf[b] else ()
        got.add((int(t.level[b]), tuple(t.coord[b]), bool(t.is_leaf[b]), pts))
    assert got == boxes
    key = lambda b: (int(t.level[b]), tuple(t.coord[b]))
    got_rel = set()
    for b in range(t.n_boxes):
        for c in t.colleagues[b]:
            if c != b and key(b) < key(c):
                got_rel.add(("colleague", key(b), key(c)))
        for c in t.coarse[b]:
            got_rel.add(("coarse", key(b), key(c)))
        for c in t.fine[b]:
            got_rel.add(("fine", key(b), key(c)))
    assert got_rel == rel


def _geom_touch(t, a, b):
    """Closed boxes intersect, tested with float box corners (tolerance 1e-9 side)."""
    ca, cb = t.box_center(a), t.box_center(b)
    ha, hb = t.box_side(a) / 2, t.box_side(b) / 2
    eps = 1e-9 * t.side
    return bool(np.all(np.abs(ca - cb) <= ha + hb + eps))


@pytest.mark.parametrize("dim,n,b", [(2, 3000, 12), (3, 3000, 16)])
def test_tree_invariants(dim, n, b):
    x = _clustered(n, dim, 3)
    t = otree.Tree(x, b)
    # every point in exactly one leaf, leaves non-empty and <= b points
    seen = np.zeros(x.shape[0], dtype=int)
    for l in t.leaves():
        assert 0 < len(t.points[l]) <= b
        seen[t.points[l]] += 1
    assert np.all(seen == 1)
    # points lie inside their leaf (float containment)
    for l in t.leaves():
        c, h = t.box_center(l), t.box_side(l) / 2
        assert np.all(np.abs(x[t.points[l]] - c) <= h * (1 + 1e-9))
    # parent / child consistency, children one level down inside the parent
    for bx in range(1, t.n_boxes):
        p = t.parent[bx]
        assert bx in t.children[p] and t.level[bx] == t.level[p] + 1
        assert all((2 * t.coord[p][d]) <= t.coord[bx][d] <= 2 * t.coord[p][d] + 1 for d in range(dim))
    # 2:1 balance: no leaf touches a box two or more levels finer
    for l in t.leaves():
        for other in range(t.n_boxes):
            if t.level[other] >= t.level[l] + 2:
                assert not _geom_touch(t, l, other)
    # neighbor lists vs the float geometric test (brute force over all boxes)
    for bx in range(t.n_boxes):
        coll = sorted(o for o in range(t.n_boxes) if t.level[o] == t.level[bx] and _geom_touch(t, bx, o))
        assert t.colleagues[bx] == coll
        assert len(coll) <= 3 ** dim and bx in coll
        coarse = sorted(o for o in range(t.n_boxes)
                        if t.level[o] == t.level[bx] - 1 and t.is_leaf[o] and _geom_touch(t, bx, o))
        assert t.coarse[bx] == coarse
        if t.is_leaf[bx]:
            fine = sorted(o for o in range(t.n_boxes) if t.level[o] == t.level[bx] + 1 and _geom_touch(t, bx, o))
            assert t.fine[bx] == fine
        else:
            assert t.fine[bx] == []
    # coarse and fine are inverse relations
    for bx in range(t.n_boxes):
        for c in t.coarse[bx]:
            assert bx in t.fine[c]
    assert sum(len(c) for c in t.coarse) > 0    # the input is adaptive


@pytest.mark.parametrize("dim", [2, 3])
def test_near_field_covered_once(dim):
    """Every pair of touching leaves is reached by exactly one translation
    route: same level (colleague path) or one level apart (coarse / fine)."""
    t = otree.Tree(_clustered(1500, dim, 5), 8)
    leaves = t.leaves()
    for a in leaves:
        for b in leaves:
            if not _geom_touch(t, a, b):
                continue
            la, lb = t.level[a], t.level[b]
            assert abs(la - lb) <= 1
            if la == lb:
                assert b in t.colleagues[a]
            elif lb == la - 1:
                assert b in t.coarse[a]
            else:
                assert b in t.fine[a]


def test_single_leaf_root():
    x = W.points_uniform(20, 3, 0)
    t = otree.Tree(x, 32)
    assert t.n_boxes == 1 and t.n_levels == 0 and t.is_leaf[0]
