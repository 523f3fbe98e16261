"""Adaptive quad/oct-tree, 2:1 balance and neighbor lists (Section 3.1).

Oracle (test infrastructure only). Brute force wherever possible so that a
reader can check each rule against the paper:

* Root: the bounding cube of the points (side = largest extent times
  (1 + 1e-12), centred on the bounding-box centre; the paper leaves the root
  unspecified).
* Split a box into 2^d children while it holds more than b points; empty
  children are pruned (Section 3.1). A point exactly on a split plane goes to
  the upper child. A box at ``MAX_DEPTH`` is never split.
* 2:1 balance (Section 3.1): a leaf may not touch any box that is two or more
  levels finer. The paper states the rule for adjacent leaves; with empty
  boxes pruned, a tree box can touch a leaf while none of its own leaves
  does, and none of the three translation types (colleague, coarse, fine)
  would then cover that pair, so the rule is applied to every box touching a
  leaf. Violating leaves are split until none is left (the least balanced
  refinement, which is unique).
* "Touching" = the closed boxes intersect (share a face, edge or corner).
* Colleagues of B: boxes on B's level touching B, B included (at most 3^d).
  Coarse neighbors of B: leaves one level up touching B. Fine neighbors of a
  leaf L: boxes one level down touching L (Section 3.1, Table of Section 3.3).

Boxes are numbered by (level, Morton key); children are ordered by child
index sum_d bit_d 2^d with x the lowest bit.
"""
from __future__ import annotations

import numpy as np

MAX_DEPTH = {2: 31, 3: 21}


def root_geometry(x: np.ndarray):
    """Centre, side and lower corner of the root box."""
    lo = x.min(axis=0)
    hi = x.max(axis=0)
    center = (lo + hi) * 0.5
    side = float(np.max(hi - lo)) * (1.0 + 1e-12)
    if side == 0.0:
        side = 1.0
    corner = center - side * 0.5
    return center, side, corner


def integer_coords(x: np.ndarray, corner: np.ndarray, side: float, depth: int) -> np.ndarray:
    """Cell index of every point on the finest grid (2^depth cells per axis)."""
    t = (x - corner) / side
    i = np.floor(t * float(2 ** depth)).astype(np.int64)
    return np.clip(i, 0, 2 ** depth - 1)


def morton_key(coord, dim: int) -> int:
    key = 0
    for bit in range(32):
        for d in range(dim):
            key |= ((int(coord[d]) >> bit) & 1) << (bit * dim + d)
    return key


def touches(la: int, ca, lb: int, cb) -> bool:
    """Closed boxes (la, ca) and (lb, cb) intersect."""
    if la > lb:
        la, ca, lb, cb = lb, cb, la, ca
    s = lb - la
    for a, b in zip(ca, cb):
        a_lo = int(a) << s
        a_hi = (int(a) + 1) << s
        if not (int(b) <= a_hi and a_lo <= int(b) + 1):
            return False
    return True


class Tree:
    """Balanced adaptive tree with neighbor lists.

    Attributes (per box id, boxes sorted by (level, Morton key)):
      level[i], coord[i] (tuple), parent[i] (-1 for the root),
      children[i] (list of box ids, child-index order), is_leaf[i],
      points[i] (sorted point indices, leaves only),
      colleagues[i], coarse[i], fine[i] (sorted box ids).
    """

    def __init__(self, x: np.ndarray, leaf_size: int):
        x = np.asarray(x, dtype=np.float64)
        self.x = x
        self.n, self.dim = x.shape
        self.leaf_size = int(leaf_size)
        self.depth = MAX_DEPTH[self.dim]
        self.center, self.side, self.corner = root_geometry(x)
        self.icoord = integer_coords(x, self.corner, self.side, self.depth)
        self._build()

    # -- construction -------------------------------------------------
    def _child_of(self, idx: np.ndarray, level: int):
        """Split point set idx of a box at `level` by child index."""
        shift = self.depth - level - 1
        bits = (self.icoord[idx] >> shift) & 1
        cidx = np.zeros(idx.shape[0], dtype=np.int64)
        for d in range(self.dim):
            cidx |= bits[:, d] << d
        out = []
        for c in range(2 ** self.dim):
            sel = idx[cidx == c]
            if sel.shape[0]:
                out.append((c, sel))
        return out

    def _build(self):
        dim = self.dim
        # node: dict(level, coord, points (if leaf), children {cidx: node})
        root = {"level": 0, "coord": (0,) * dim, "points": np.arange(self.n), "children": None}
        stack = [root]
        while stack:
            node = stack.pop()
            pts = node["points"]
            if pts.shape[0] > self.leaf_size and node["level"] < self.depth:
                self._split(node)
                stack.extend(node["children"].values())
        # 2:1 balance: split every leaf touched by a box two or more levels finer
        while True:
            nodes = self._all_nodes(root)
            levels = np.array([n["level"] for n in nodes])
            coords = np.array([n["coord"] for n in nodes], dtype=np.int64)
            violators = []
            for nd in nodes:
                if nd["children"] is not None:
                    continue
                fine = np.nonzero(levels >= nd["level"] + 2)[0]
                if fine.shape[0] == 0:
                    continue
                s = levels[fine] - nd["level"]
                lo = np.array(nd["coord"], dtype=np.int64)[None, :] << s[:, None]
                hi = (np.array(nd["coord"], dtype=np.int64)[None, :] + 1) << s[:, None]
                c = coords[fine]
                hit = np.all((c <= hi) & (lo <= c + 1), axis=1)
                if np.any(hit):
                    violators.append(nd)
            if not violators:
                break
            for nd in violators:
                self._split(nd)
        self._number(root)

    def _split(self, node):
        children = {}
        for c, sel in self._child_of(node["points"], node["level"]):
            coord = tuple(2 * node["coord"][d] + ((c >> d) & 1) for d in range(self.dim))
            children[c] = {"level": node["level"] + 1, "coord": coord, "points": sel, "children": None}
        node["children"] = children

    @staticmethod
    def _all_nodes(root):
        out, stack = [], [root]
        while stack:
            nd = stack.pop()
            out.append(nd)
            if nd["children"] is not None:
                stack.extend(nd["children"].values())
        return out

    def _number(self, root):
        nodes = self._all_nodes(root)
        nodes.sort(key=lambda nd: (nd["level"], morton_key(nd["coord"], self.dim)))
        for i, nd in enumerate(nodes):
            nd["id"] = i
        nb = len(nodes)
        self.n_boxes = nb
        self.level = np.array([nd["level"] for nd in nodes], dtype=np.int64)
        self.coord = [nd["coord"] for nd in nodes]
        self.parent = np.full(nb, -1, dtype=np.int64)
        self.children = [[] for _ in range(nb)]
        self.is_leaf = np.zeros(nb, dtype=bool)
        self.points = [None] * nb
        for nd in nodes:
            i = nd["id"]
            if nd["children"] is None:
                self.is_leaf[i] = True
                self.points[i] = np.sort(nd["points"])
            else:
                for c in sorted(nd["children"]):
                    ch = nd["children"][c]["id"]
                    self.children[i].append(ch)
                    self.parent[ch] = i
        self.n_levels = int(self.level.max())
        self.boxes_at = [np.nonzero(self.level == l)[0] for l in range(self.n_levels + 1)]
        self._neighbors()

    def touching(self, i: int) -> np.ndarray:
        """Ids of all boxes within one level of box i whose closed box touches it."""
        li = int(self.level[i])
        lv = self.level
        cand = np.nonzero(np.abs(lv - li) <= 1)[0]
        cc = self._coord_arr[cand]
        ci = self._coord_arr[i][None, :]
        lc = lv[cand][:, None]
        # scale the coarser of the two boxes to the finer level, closed intervals
        fine_lvl = np.maximum(lc, li)
        s_i = fine_lvl - li
        s_c = fine_lvl - lc
        i_lo, i_hi = ci << s_i, (ci + 1) << s_i
        c_lo, c_hi = cc << s_c, (cc + 1) << s_c
        hit = np.all((c_lo <= i_hi) & (i_lo <= c_hi), axis=1)
        return cand[hit]

    def _neighbors(self):
        nb = self.n_boxes
        self._coord_arr = np.array(self.coord, dtype=np.int64)
        self.colleagues = [[] for _ in range(nb)]
        self.coarse = [[] for _ in range(nb)]
        self.fine = [[] for _ in range(nb)]
        for i in range(nb):
            li = int(self.level[i])
            for j in self.touching(i):
                lj = int(self.level[j])
                if lj == li:
                    self.colleagues[i].append(int(j))
                elif lj == li - 1 and self.is_leaf[j]:
                    self.coarse[i].append(int(j))
                elif lj == li + 1 and self.is_leaf[i]:
                    self.fine[i].append(int(j))

    # -- geometry -----------------------------------------------------
    def box_side(self, i: int) -> float:
        return self.side / float(2 ** int(self.level[i]))

    def box_center(self, i: int) -> np.ndarray:
        a = self.box_side(i)
        return self.corner + (np.array(self.coord[i], dtype=np.float64) + 0.5) * a

    def leaves(self):
        return [i for i in range(self.n_boxes) if self.is_leaf[i]]
