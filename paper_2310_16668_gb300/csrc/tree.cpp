// Adaptive quad/oct-tree with 2:1 balance and neighbor lists (Section 3.1).
//
// * Root: bounding cube of the points, side = largest extent * (1 + 1e-12),
//   centred on the bounding-box centre.
// * Every point gets integer cell coordinates on the finest grid
//   (2^D cells per axis, D = 31 in 2D, 21 in 3D); the box containing it at
//   level l is those coordinates shifted right by D - l, so a point on a split
//   plane belongs to the upper child.
// * Boxes holding more than b points are split into their non-empty children.
// * 2:1 balance: a leaf may not touch any box two or more levels finer. Every
//   such leaf is split until none is left; this is the least balanced
//   refinement, so the result does not depend on the order of the splits.
// * Colleagues (same level, touching, self included), coarse neighbors
//   (leaves one level up touching the box) and fine neighbors (boxes one level
//   down touching a leaf).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_map>
#include <unordered_set>

#include "host.h"

namespace skel {

namespace {

uint64_t interleave(const int64_t* c, int dim) {
    uint64_t key = 0;
    for (int bit = 0; bit < (dim == 2 ? 32 : 21); ++bit)
        for (int d = 0; d < dim; ++d)
            key |= (uint64_t)((c[d] >> bit) & 1) << (bit * dim + d);
    return key;
}

struct TmpBox {
    int level;
    uint64_t key;                 // Morton key at its own level
    int64_t lo, hi;               // range in the Morton-sorted point order
    bool leaf;
};

struct LevelMap {
    std::vector<std::unordered_map<uint64_t, int64_t>> m;   // per level: key -> TmpBox index
    int64_t find(int l, uint64_t key) const {
        if (l < 0 || l >= (int)m.size()) return -1;
        auto it = m[l].find(key);
        return it == m[l].end() ? -1 : it->second;
    }
};

}  // namespace

bool touches(int la, const int64_t* ca, int lb, const int64_t* cb, int dim) {
    if (la > lb) { std::swap(la, lb); std::swap(ca, cb); }
    int s = lb - la;
    for (int d = 0; d < dim; ++d) {
        int64_t a_lo = ca[d] << s, a_hi = (ca[d] + 1) << s;
        if (!(cb[d] <= a_hi && a_lo <= cb[d] + 1)) return false;
    }
    return true;
}

void build_tree(const double* X, int64_t n, int dim, int b, Tree& t,
                std::vector<std::vector<int64_t>>& leaf_points) {
    const int D = max_depth(dim);
    t.dim = dim;
    t.n = n;
    double lo[3], hi[3];
    for (int d = 0; d < dim; ++d) { lo[d] = X[d]; hi[d] = X[d]; }
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < dim; ++d) {
            lo[d] = std::min(lo[d], X[i * dim + d]);
            hi[d] = std::max(hi[d], X[i * dim + d]);
        }
    double ext = 0;
    for (int d = 0; d < dim; ++d) {
        t.center[d] = (lo[d] + hi[d]) * 0.5;
        ext = std::max(ext, hi[d] - lo[d]);
    }
    t.side = ext * (1.0 + 1e-12);
    if (t.side == 0.0) t.side = 1.0;
    for (int d = 0; d < dim; ++d) t.corner[d] = t.center[d] - t.side * 0.5;

    const double scale = std::ldexp(1.0, D);
    const int64_t cmax = ((int64_t)1 << D) - 1;
    std::vector<uint64_t> key(n);
    {
        int64_t c[3];
        for (int64_t i = 0; i < n; ++i) {
            for (int d = 0; d < dim; ++d) {
                double tt = (X[i * dim + d] - t.corner[d]) / t.side;
                int64_t v = (int64_t)std::floor(tt * scale);
                c[d] = std::min(std::max(v, (int64_t)0), cmax);
            }
            key[i] = interleave(c, dim);
        }
    }
    std::vector<int64_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
        return key[a] < key[c] || (key[a] == key[c] && a < c);
    });
    std::vector<uint64_t> skey(n);
    for (int64_t i = 0; i < n; ++i) skey[i] = key[order[i]];

    std::vector<TmpBox> boxes;
    LevelMap lm;
    lm.m.resize(D + 1);
    auto add_box = [&](int l, uint64_t k, int64_t a, int64_t c, bool leaf) {
        boxes.push_back({l, k, a, c, leaf});
        lm.m[l][k] = (int64_t)boxes.size() - 1;
        return (int64_t)boxes.size() - 1;
    };
    const uint64_t cmask = ((uint64_t)1 << dim) - 1;
    // split box bi into its non-empty children; returns their indices
    auto split = [&](int64_t bi, std::vector<int64_t>* out) {
        TmpBox B = boxes[bi];
        boxes[bi].leaf = false;
        int shift = (D - B.level - 1) * dim;
        int64_t a = B.lo;
        while (a < B.hi) {
            uint64_t c = (skey[a] >> shift) & cmask;
            int64_t e = a;
            while (e < B.hi && ((skey[e] >> shift) & cmask) == c) ++e;
            int64_t id = add_box(B.level + 1, (B.key << dim) | c, a, e, true);
            if (out) out->push_back(id);
            a = e;
        }
    };
    add_box(0, 0, 0, n, true);
    {
        std::vector<int64_t> stack{0};
        while (!stack.empty()) {
            int64_t bi = stack.back();
            stack.pop_back();
            if (boxes[bi].hi - boxes[bi].lo > b && boxes[bi].level < D) split(bi, &stack);
        }
    }
    // 2:1 balance (least fixed point)
    auto decode = [&](uint64_t k, int64_t* c) {
        for (int d = 0; d < dim; ++d) c[d] = 0;
        for (int bit = 0; bit < (dim == 2 ? 32 : 21); ++bit)
            for (int d = 0; d < dim; ++d) c[d] |= (int64_t)((k >> (bit * dim + d)) & 1) << bit;
    };
    const int noff = dim == 2 ? 9 : 27;
    while (true) {
        std::unordered_set<int64_t> viol;
        for (size_t bi = 0; bi < boxes.size(); ++bi) {
            const TmpBox& B = boxes[bi];
            if (B.level < 2) continue;
            int64_t c[3], p[3], pm[3];
            decode(B.key, c);
            const int64_t ncell = (int64_t)1 << B.level;
            for (int o = 0; o < noff; ++o) {
                int oo = o;
                bool ok = true, zero = true;
                for (int d = 0; d < dim; ++d) {
                    int off = oo % 3 - 1;
                    oo /= 3;
                    p[d] = c[d] + off;
                    if (off != 0) zero = false;
                    if (p[d] < 0 || p[d] >= ncell) ok = false;
                }
                if (!ok || zero) continue;
                for (int m = B.level - 1; m >= 0; --m) {
                    for (int d = 0; d < dim; ++d) pm[d] = p[d] >> (B.level - m);
                    int64_t f = lm.find(m, interleave(pm, dim));
                    if (f >= 0) {
                        if (boxes[f].leaf && m <= B.level - 2) viol.insert(f);
                        break;
                    }
                }
            }
        }
        if (viol.empty()) break;
        std::vector<int64_t> vs(viol.begin(), viol.end());
        std::sort(vs.begin(), vs.end());
        for (int64_t f : vs) split(f, nullptr);
    }
    // number boxes by (level, Morton key)
    std::vector<int64_t> ord(boxes.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t c) {
        return boxes[a].level < boxes[c].level ||
               (boxes[a].level == boxes[c].level && boxes[a].key < boxes[c].key);
    });
    const int64_t nb = (int64_t)boxes.size();
    t.nb = nb;
    t.level.resize(nb);
    t.coord.resize(nb * dim);
    t.parent.assign(nb, -1);
    t.is_leaf.resize(nb);
    leaf_points.assign(nb, {});
    std::vector<int64_t> newid(nb);
    for (int64_t i = 0; i < nb; ++i) newid[ord[i]] = i;
    for (int64_t i = 0; i < nb; ++i) {
        const TmpBox& B = boxes[ord[i]];
        t.level[i] = B.level;
        decode(B.key, &t.coord[i * dim]);
        t.is_leaf[i] = B.leaf ? 1 : 0;
        if (B.level > 0) t.parent[i] = newid[lm.find(B.level - 1, B.key >> dim)];
        if (B.leaf) {
            std::vector<int64_t>& lp = leaf_points[i];
            lp.assign(order.begin() + B.lo, order.begin() + B.hi);
            std::sort(lp.begin(), lp.end());
        }
    }
    finish_tree(t);
}

void finish_tree(Tree& t) {
    const int dim = t.dim;
    const int64_t nb = t.nb;
    t.L = 0;
    for (int64_t i = 0; i < nb; ++i) t.L = std::max(t.L, (int)t.level[i]);
    t.level_ptr.assign(t.L + 2, 0);
    for (int64_t i = 0; i < nb; ++i) t.level_ptr[t.level[i] + 1]++;
    for (int l = 0; l <= t.L; ++l) t.level_ptr[l + 1] += t.level_ptr[l];
    // children (boxes are sorted by (level, key), so children come in key order)
    t.child_ptr.assign(nb + 1, 0);
    for (int64_t i = 0; i < nb; ++i)
        if (t.parent[i] >= 0) t.child_ptr[t.parent[i] + 1]++;
    for (int64_t i = 0; i < nb; ++i) t.child_ptr[i + 1] += t.child_ptr[i];
    t.child.assign(t.child_ptr[nb], 0);
    {
        std::vector<int64_t> fill(t.child_ptr.begin(), t.child_ptr.end() - 1);
        for (int64_t i = 0; i < nb; ++i)
            if (t.parent[i] >= 0) t.child[fill[t.parent[i]]++] = i;
    }
    // lookup (level, key) -> box
    std::vector<std::unordered_map<uint64_t, int64_t>> lm(t.L + 1);
    for (int64_t i = 0; i < nb; ++i) lm[t.level[i]][interleave(&t.coord[i * dim], dim)] = i;
    auto find = [&](int l, const int64_t* c) -> int64_t {
        if (l < 0 || l > t.L) return -1;
        const int64_t ncell = (int64_t)1 << l;
        for (int d = 0; d < dim; ++d)
            if (c[d] < 0 || c[d] >= ncell) return -1;
        auto it = lm[l].find(interleave(c, dim));
        return it == lm[l].end() ? -1 : it->second;
    };
    const int noff = dim == 2 ? 9 : 27;
    std::vector<std::vector<int64_t>> coll(nb), coarse(nb), fine(nb);
    for (int64_t i = 0; i < nb; ++i) {
        const int l = t.level[i];
        const int64_t* c = &t.coord[i * dim];
        int64_t p[3], pp[3];
        for (int o = 0; o < noff; ++o) {
            int oo = o;
            bool zero = true;
            for (int d = 0; d < dim; ++d) {
                int off = oo % 3 - 1;
                oo /= 3;
                p[d] = c[d] + off;
                if (off) zero = false;
            }
            int64_t j = find(l, p);
            if (j >= 0) coll[i].push_back(j);
            if (!zero && l >= 1) {
                bool inb = true;
                for (int d = 0; d < dim; ++d) {
                    if (p[d] < 0 || p[d] >= ((int64_t)1 << l)) inb = false;
                    pp[d] = p[d] >> 1;
                }
                if (inb) {
                    int64_t f = find(l - 1, pp);
                    if (f >= 0 && t.is_leaf[f]) coarse[i].push_back(f);
                }
            }
        }
    }
    for (int64_t i = 0; i < nb; ++i) {
        std::sort(coll[i].begin(), coll[i].end());
        std::sort(coarse[i].begin(), coarse[i].end());
        coarse[i].erase(std::unique(coarse[i].begin(), coarse[i].end()), coarse[i].end());
    }
    for (int64_t i = 0; i < nb; ++i) {
        if (!t.is_leaf[i]) continue;
        for (int64_t cj : coll[i]) {
            if (cj == i || t.is_leaf[cj]) continue;
            for (int64_t q = t.child_ptr[cj]; q < t.child_ptr[cj + 1]; ++q) {
                int64_t ch = t.child[q];
                if (touches(t.level[i], &t.coord[i * dim], t.level[ch], &t.coord[ch * dim], dim))
                    fine[i].push_back(ch);
            }
        }
        std::sort(fine[i].begin(), fine[i].end());
    }
    auto to_csr = [&](std::vector<std::vector<int64_t>>& v, std::vector<int64_t>& ptr,
                      std::vector<int64_t>& lst) {
        ptr.assign(nb + 1, 0);
        for (int64_t i = 0; i < nb; ++i) ptr[i + 1] = ptr[i] + (int64_t)v[i].size();
        lst.clear();
        lst.reserve(ptr[nb]);
        for (int64_t i = 0; i < nb; ++i) lst.insert(lst.end(), v[i].begin(), v[i].end());
    };
    to_csr(coll, t.coll_ptr, t.coll);
    to_csr(coarse, t.coarse_ptr, t.coarse);
    to_csr(fine, t.fine_ptr, t.fine);
}

}  // namespace skel
