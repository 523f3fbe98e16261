// Flattened device layout of Algorithm 2 with the translations regrouped.
//
// Entry space: every box B on levels >= top (top = 1, or 0 when the root is
// the only box) owns a contiguous segment of |I_B| entries in slot order, so
// a tree box's segment is its children's skeletons back to back. The upward
// pass writes qhat_{S_c} of child c straight into slot c of its parent's
// segment (the concatenation of Algorithm 2 is free), and the downward pass
// reads uhat_{S_c} from the same place.
//
// Near field. Algorithm 2 adds u_B += A_{B,B_j} q_{B_j} over colleagues and,
// one level down, subtracts uhat_{S_c} -= A_{S_c,S_c'} qhat_{S_c'} over
// colleague children c, c'. Both write the same entries of level l's entry
// space (uhat_{S_c} lives in slot c of the parent), and qhat_{S_c'} is slot
// c' of the colleague's segment, so the subtraction cancels exactly the
// (c, c') block of the addition. The layout therefore evaluates every
// colleague block once with the touching child pairs masked out (a 64-bit
// mask per task, bit c*8 + c'). The ifs and tfo subtractions cancel blocks
// the same way (a child touching a colleague leaf; a colleague's child
// touching a leaf), and their additions become unmasked tasks between
// levels. The sums are regrouped, never approximated.
//
// Tasks between two touching leaves are flagged TASK_ADJ: only they can hold
// arbitrarily close (or coincident) pairs.
#include <algorithm>
#include <numeric>

#include "host.h"

namespace skel {

namespace {
constexpr int64_t kItemCost = 2048;   // source entries per warp work item
}

// class of a tile-list length: lengths within a factor 1.25 share a class
int length_class(int n) {
    int c = 0;
    for (double v = 1.0; v * 1.25 <= (double)n; v *= 1.25) ++c;
    return c;
}

void build_layout(const Plan& p, Layout& lay) {
    const Tree& t = p.tree;
    const Skel& sk = p.sk;
    const int dim = t.dim;
    const int64_t nb = t.nb;
    lay.top = t.L >= 1 ? 1 : 0;

    // ---- entry space ----------------------------------------------------
    lay.box_off.assign(nb, -1);
    lay.box_n.assign(nb, 0);
    lay.box_nslot.assign(nb, 0);
    lay.slot_start.assign(nb * (kMaxSlots + 1), 0);
    int64_t off = 0;
    for (int64_t b = 0; b < nb; ++b) {
        if (t.level[b] < lay.top) continue;
        const int64_t n = sk.idx_ptr[b + 1] - sk.idx_ptr[b];
        lay.box_off[b] = off;
        lay.box_n[b] = (int32_t)n;
        off += n;
        int32_t* ss = &lay.slot_start[b * (kMaxSlots + 1)];
        if (t.is_leaf[b]) {
            lay.box_nslot[b] = 1;
            ss[0] = 0;
            ss[1] = (int32_t)n;
        } else {
            int s = 0;
            int32_t acc = 0;
            for (int64_t q = t.child_ptr[b]; q < t.child_ptr[b + 1]; ++q, ++s) {
                ss[s] = acc;
                acc += sk.k[t.child[q]];
            }
            ss[s] = acc;
            lay.box_nslot[b] = s;
            if (acc != n) throw Error(-1, "layout: index set is not the children's skeletons");
        }
    }
    lay.n_tot = off;
    lay.X.assign(lay.n_tot * 4, 0.0);
    lay.pos.assign(lay.n_tot, 0);
    lay.perm_entry.clear();
    lay.perm_point.clear();
    for (int64_t b = 0; b < nb; ++b) {
        if (lay.box_off[b] < 0) continue;
        const int64_t o = lay.box_off[b];
        for (int64_t i = 0; i < lay.box_n[b]; ++i) {
            const int64_t pt = sk.idx[sk.idx_ptr[b] + i];
            for (int d = 0; d < dim; ++d) lay.X[(o + i) * 4 + d] = p.pts[pt * dim + d];
            lay.pos[o + i] = (int32_t)sk.piv[sk.idx_ptr[b] + i];
            if (t.is_leaf[b]) {
                lay.perm_entry.push_back(o + i);
                lay.perm_point.push_back(pt);
            }
        }
    }

    // ---- upward / downward boxes -----------------------------------------
    const int lo_up = std::max(2, lay.top + 1);
    lay.up.clear();
    lay.up_leaf.clear();
    lay.up_level_ptr.assign(t.L + 2, 0);
    for (int l = 0; l <= t.L; ++l) {
        lay.up_level_ptr[l] = (int64_t)lay.up.size();
        if (l < lo_up) continue;
        for (int64_t b = t.level_ptr[l]; b < t.level_ptr[l + 1]; ++b) {
            const int64_t par = t.parent[b];
            int s = 0;
            for (int64_t q = t.child_ptr[par]; q < t.child_ptr[par + 1]; ++q, ++s)
                if (t.child[q] == b) break;
            UpBox u;
            u.off = lay.box_off[b];
            u.dst = lay.box_off[par] + lay.slot_start[par * (kMaxSlots + 1) + s];
            u.T_off = sk.T_ptr[b];
            u.n = lay.box_n[b];
            u.k = sk.k[b];
            lay.up.push_back(u);
            lay.up_leaf.push_back(t.is_leaf[b] ? 1 : 0);
        }
    }
    lay.up_level_ptr[t.L + 1] = (int64_t)lay.up.size();
    lay.T = sk.T;

    // ---- near-field tasks ---------------------------------------------------
    auto child_of = [&](int64_t b, int s) { return t.child[t.child_ptr[b] + s]; };
    auto C = [&](int64_t b) { return &t.coord[b * dim]; };
    lay.task_ptr.assign(nb + 1, 0);
    lay.task_src.clear();
    lay.task_mask.clear();
    lay.task_flags.clear();
    lay.pairs_direct = lay.pairs_far = 0;
    auto slot_size = [&](int64_t b, int s) {
        const int32_t* ss = &lay.slot_start[b * (kMaxSlots + 1)];
        return (int64_t)(ss[s + 1] - ss[s]);
    };
    auto add_task = [&](int64_t b, int64_t src, uint64_t mask, int32_t flags) {
        lay.task_src.push_back(src);
        lay.task_mask.push_back(mask);
        lay.task_flags.push_back(flags);
        for (int i = 0; i < lay.box_nslot[b]; ++i)
            for (int j = 0; j < lay.box_nslot[src]; ++j)
                if (!((mask >> (i * 8 + j)) & 1)) {
                    int64_t pr = slot_size(b, i) * slot_size(src, j);
                    if (flags & TASK_ADJ) lay.pairs_direct += pr; else lay.pairs_far += pr;
                }
    };
    for (int64_t b = 0; b < nb; ++b) {
        lay.task_ptr[b] = (int64_t)lay.task_src.size();
        if (lay.box_off[b] < 0) continue;
        const int l = t.level[b];
        const bool bl = t.is_leaf[b];
        for (int64_t q = t.coll_ptr[b]; q < t.coll_ptr[b + 1]; ++q) {
            const int64_t bj = t.coll[q];
            const bool jl = t.is_leaf[bj];
            uint64_t mask = 0;
            int32_t flags = 0;
            if (bl && jl) {
                flags = TASK_ADJ;
            } else if (!bl && !jl) {
                for (int i = 0; i < lay.box_nslot[b]; ++i)
                    for (int j = 0; j < lay.box_nslot[bj]; ++j) {
                        const int64_t ci = child_of(b, i), cj = child_of(bj, j);
                        if (touches(l + 1, C(ci), l + 1, C(cj), dim)) mask |= (uint64_t)1 << (i * 8 + j);
                    }
            } else if (!bl && jl) {
                for (int i = 0; i < lay.box_nslot[b]; ++i)
                    if (touches(l + 1, C(child_of(b, i)), l, C(bj), dim)) mask |= (uint64_t)1 << (i * 8);
            } else {
                for (int j = 0; j < lay.box_nslot[bj]; ++j)
                    if (touches(l, C(b), l + 1, C(child_of(bj, j)), dim)) mask |= (uint64_t)1 << j;
            }
            add_task(b, bj, mask, flags);
        }
        if (l > lay.top)
            for (int64_t q = t.coarse_ptr[b]; q < t.coarse_ptr[b + 1]; ++q)
                add_task(b, t.coarse[q], 0, bl ? TASK_ADJ : 0);
        if (bl)
            for (int64_t q = t.fine_ptr[b]; q < t.fine_ptr[b + 1]; ++q)
                add_task(b, t.fine[q], 0, t.is_leaf[t.fine[q]] ? TASK_ADJ : 0);
    }
    lay.task_ptr[nb] = (int64_t)lay.task_src.size();

    // ---- warp work items: 32 targets x a range of tasks ---------------------
    // every partial sum is (slot, row): slot = one work item's 32-row block;
    // per entry, the list of partial sums that add up to its translations
    std::vector<std::pair<int64_t, int64_t>> parts;             // (entry, slot * 32 + row)
    auto to_csr = [&](std::vector<std::pair<int64_t, int64_t>>& ps, std::vector<int64_t>& ptr,
                      std::vector<int64_t>& idx) {
        std::stable_sort(ps.begin(), ps.end(), [](const std::pair<int64_t, int64_t>& a,
                                                  const std::pair<int64_t, int64_t>& c) { return a.first < c.first; });
        ptr.assign(lay.n_tot + 1, 0);
        for (auto& x : ps) ptr[x.first + 1]++;
        for (int64_t e = 0; e < lay.n_tot; ++e) ptr[e + 1] += ptr[e];
        idx.resize(ps.size());
        for (size_t i = 0; i < ps.size(); ++i) idx[i] = ps[i].second;
        ps.clear();
    };
    struct Tmp { WorkItem it; int64_t cost; };
    auto simt_items = [&](auto use_box, std::vector<WorkItem>& out, int64_t slot0) {
        std::vector<Tmp> tmp;
        for (int64_t b = 0; b < nb; ++b) {
            if (lay.box_off[b] < 0 || !use_box(b)) continue;
            const int32_t* ss = &lay.slot_start[b * (kMaxSlots + 1)];
            for (int32_t t0 = 0; t0 < lay.box_n[b]; t0 += kChunk) {
                const int32_t t1 = std::min(t0 + kChunk, lay.box_n[b]);
                uint32_t slots = 0;
                for (int i = 0; i < lay.box_nslot[b]; ++i)
                    if (ss[i] < t1 && ss[i + 1] > t0) slots |= 1u << i;
                int64_t lo = lay.task_ptr[b], cost = 0;
                for (int64_t tk = lay.task_ptr[b]; tk < lay.task_ptr[b + 1]; ++tk) {
                    const int64_t src = lay.task_src[tk];
                    int64_t c = 0;
                    for (int j = 0; j < lay.box_nslot[src]; ++j) {
                        bool any = false;
                        for (int i = 0; i < lay.box_nslot[b]; ++i)
                            if (((slots >> i) & 1) && !((lay.task_mask[tk] >> (i * 8 + j)) & 1)) any = true;
                        if (any) c += slot_size(src, j);
                    }
                    if (cost > 0 && cost + c > kItemCost) {
                        tmp.push_back({{b, t0, (int32_t)lo, (int32_t)tk, 0}, cost});
                        lo = tk;
                        cost = 0;
                    }
                    cost += c;
                }
                tmp.push_back({{b, t0, (int32_t)lo, (int32_t)lay.task_ptr[b + 1], 0}, cost});
            }
        }
        std::vector<int64_t> order(tmp.size());
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int64_t a, int64_t c) { return tmp[a].cost > tmp[c].cost; });
        out.resize(tmp.size());
        for (size_t r = 0; r < order.size(); ++r) {
            const WorkItem& it = tmp[order[r]].it;
            out[r] = it;
            const int32_t t1 = std::min(it.t0 + kChunk, lay.box_n[it.tgt_box]);
            for (int32_t t = it.t0; t < t1; ++t)
                parts.push_back({lay.box_off[it.tgt_box] + t, (slot0 + (int64_t)r) * kChunk + (t - it.t0)});
        }
    };
    simt_items([](int64_t) { return true; }, lay.items, 0);
    to_csr(parts, lay.part_ptr, lay.part_idx);

    // ---- tensor-core mode --------------------------------------------------------
    // tree boxes and large leaves: their own 128-row items (a small tree box
    // fills part of one: at many right-hand sides that still beats the CUDA
    // cores); small leaves: packed, consecutive in box order (so neighbouring
    // in space), up to 128 rows and 8 leaves per item, one keep-mask slot per
    // leaf. The CUDA-core list for the remaining boxes is then empty.
    auto is_tc = [&](int64_t b) { return !t.is_leaf[b] || lay.box_n[b] >= kTcMinRows; };
    auto packable = [&](int64_t b) { return !is_tc(b) && t.is_leaf[b]; };
    simt_items([&](int64_t b) { return !is_tc(b) && !packable(b); }, lay.mix_items, 0);
    int64_t slot = (int64_t)lay.mix_items.size();
    lay.tc_tiles.clear();
    lay.tc_items.clear();
    lay.pairs_tc = 0;
    lay.box_chunk0.assign(nb, -1);
    lay.chunk_start.clear();
    lay.chunk_cnt.clear();
    lay.chunk_center.clear();
    // box centres in FP32: the tensor-core path measures coordinates from the
    // source box's centre, so FP32 keeps their resolution relative to the box
    auto box_center = [&](int64_t b, int d) {
        const double h = t.side / (double)(1ll << t.level[b]);
        return (float)(t.corner[d] + ((double)t.coord[b * dim + d] + 0.5) * h);
    };
    for (int64_t b = 0; b < nb; ++b) {
        if (lay.box_off[b] < 0) continue;
        lay.box_chunk0[b] = (int64_t)lay.chunk_start.size();
        for (int32_t p0 = 0; p0 < lay.box_n[b]; p0 += kTcK) {
            lay.chunk_start.push_back(lay.box_off[b] + p0);
            lay.chunk_cnt.push_back(std::min(kTcK, lay.box_n[b] - p0));
            for (int d = 0; d < 4; ++d) lay.chunk_center.push_back(d < dim ? box_center(b, d) : 0.f);
        }
    }
    // one item: rows [row_off, row_off + nrows) whose slot j covers rows
    // [sst[j], sst[j+1]); targets = (box, first slot of that box in the item,
    // row of the box's first entry)
    struct Tgt { int64_t box; int slot0; int32_t row0; };
    auto emit = [&](int64_t row_off, int32_t nrows, int nslot, const int32_t* sst, const std::vector<Tgt>& tg) {
        // the union of the targets' tasks, one tile run per (source box, flags)
        std::vector<std::pair<int64_t, int32_t>> srcs;                 // (source box, flags)
        std::vector<std::vector<uint64_t>> keepslot;                  // per source: per item slot, mask of source slots kept
        for (const Tgt& g : tg) {
            const int64_t b = g.box;
            for (int64_t tk = lay.task_ptr[b]; tk < lay.task_ptr[b + 1]; ++tk) {
                const int64_t src = lay.task_src[tk];
                size_t k = 0;
                while (k < srcs.size() && !(srcs[k].first == src && srcs[k].second == lay.task_flags[tk])) ++k;
                if (k == srcs.size()) {
                    srcs.push_back({src, lay.task_flags[tk]});
                    keepslot.push_back(std::vector<uint64_t>(kMaxSlots, 0));
                }
                for (int i = 0; i < lay.box_nslot[b]; ++i) {
                    const int is = g.slot0 + i;
                    if (is < 0 || is >= nslot) continue;
                    for (int j = 0; j < lay.box_nslot[src]; ++j)
                        if (!((lay.task_mask[tk] >> (i * 8 + j)) & 1)) keepslot[k][is] |= (uint64_t)1 << j;
                }
            }
        }
        TcItem it{};
        it.row_off = row_off;
        it.nrows = nrows;
        it.nslot = nslot;
        for (int j = 0; j <= nslot; ++j) it.slot_start[j] = sst[j];
        it.list_lo = (int32_t)lay.tc_tiles.size();
        for (size_t k = 0; k < srcs.size(); ++k) {
            const int64_t src = srcs[k].first;
            const int32_t* ssS = &lay.slot_start[src * (kMaxSlots + 1)];
            const int32_t n = lay.box_n[src];
            for (int32_t p0 = 0; p0 < n; p0 += kTcK) {
                SrcTile st{};
                st.start = lay.box_off[src] + p0;
                st.chunk = (int32_t)(lay.box_chunk0[src] + p0 / kTcK);
                for (int d = 0; d < 3; ++d) st.cen[d] = d < dim ? box_center(src, d) : 0.f;
                st.cnt = std::min(kTcK, n - p0);
                st.flags = srcs[k].second;
                for (int j = 0; j < lay.box_nslot[src]; ++j) {
                    const int a = std::max(ssS[j] - p0, 0), e = std::min(ssS[j + 1] - p0, st.cnt);
                    if (e <= a) continue;
                    const uint32_t bits = (uint32_t)(((1ull << e) - 1ull) ^ ((1ull << a) - 1ull));
                    for (int is = 0; is < nslot; ++is)
                        if ((keepslot[k][is] >> j) & 1) st.keep[is] |= bits;
                }
                bool any = false;
                for (int is = 0; is < nslot; ++is) {
                    any |= st.keep[is] != 0;
                    const int32_t rows_is = std::min(sst[is + 1], nrows) - std::max(sst[is], 0);
                    if (rows_is > 0) lay.pairs_tc += (int64_t)rows_is * __builtin_popcount(st.keep[is]);
                }
                if (!any) continue;
                lay.tc_tiles.push_back(st);
            }
        }
        // the whole list stays one item: its rows get exactly one writer
        it.list_hi = (int32_t)lay.tc_tiles.size();
        it.slot = 0;
        lay.tc_items.push_back(it);
    };
    for (int64_t b = 0; b < nb; ++b) {
        if (lay.box_off[b] < 0 || !is_tc(b)) continue;
        const int32_t* ssB = &lay.slot_start[b * (kMaxSlots + 1)];
        for (int32_t r0 = 0; r0 < lay.box_n[b]; r0 += kTcRows) {
            int32_t sst[kMaxSlots + 1];
            for (int j = 0; j <= lay.box_nslot[b]; ++j) sst[j] = ssB[j] - r0;
            emit(lay.box_off[b] + r0, std::min(kTcRows, lay.box_n[b] - r0), lay.box_nslot[b], sst,
                 {Tgt{b, 0, -r0}});
        }
    }
    for (int64_t b = 0; b < nb;) {
        if (lay.box_off[b] < 0 || !packable(b)) { ++b; continue; }
        // consecutive packable leaves with contiguous segments
        std::vector<Tgt> tg;
        int32_t sst[kMaxSlots + 1];
        int32_t rows = 0;
        const int64_t row_off = lay.box_off[b];
        while (b < nb && lay.box_off[b] >= 0 && packable(b) && (int)tg.size() < kMaxSlots &&
               rows + lay.box_n[b] <= kTcRows && lay.box_off[b] == row_off + rows) {
            sst[tg.size()] = rows;
            tg.push_back(Tgt{b, (int)tg.size(), rows});
            rows += lay.box_n[b];
            ++b;
        }
        sst[tg.size()] = rows;
        emit(row_off, rows, (int)tg.size(), sst, tg);
    }
    // longest lists first, so that the long items start early, by classes of
    // lengths within 25% of each other; within a class the items keep their
    // order (boxes in level and Morton order), so that items running at the
    // same time read the same neighbouring source chunks (L2 reuse)
    std::stable_sort(lay.tc_items.begin(), lay.tc_items.end(), [](const TcItem& a, const TcItem& c) {
        return length_class(a.list_hi - a.list_lo) > length_class(c.list_hi - c.list_lo);
    });
    // the partial sums of the CUDA-core items (small non-leaf boxes) only;
    // tensor-core items write their rows of U directly
    lay.tc_n_slots = slot;
    to_csr(parts, lay.tc_part_ptr, lay.tc_part_idx);
}

}  // namespace skel

namespace skel {

// Concatenate the layouts of independent point sets into one: every index is
// shifted by the entries, points, boxes, tasks, items, tiles, chunks and
// operator entries of the sets before it, and the up/down boxes are grouped
// by level across sets, so that each phase of the apply is one launch over
// all sets. No task, item or box refers across sets, and every per-entry sum
// keeps its order (the CSR lists are concatenated, not re-sorted), so each
// set's result is the one its own layout gives.
void merge_layouts(const std::vector<const Layout*>& ls, const std::vector<int64_t>& n_points,
                   const std::vector<int64_t>& n_boxes, int T_width, Layout& m) {
    m = Layout();
    m.top = 1;
    int Lmax = 0;
    for (const Layout* l : ls) Lmax = std::max(Lmax, (int)l->up_level_ptr.size() - 2);
    std::vector<int64_t> e0, p0, b0, k0, w0, mw0, t0, c0, T0;   // per-set offsets
    int64_t eo = 0, po = 0, bo = 0, ko = 0, wo = 0, mwo = 0, to = 0, co = 0, To = 0;
    for (size_t s = 0; s < ls.size(); ++s) {
        const Layout& l = *ls[s];
        e0.push_back(eo); p0.push_back(po); b0.push_back(bo); k0.push_back(ko);
        w0.push_back(wo); mw0.push_back(mwo); t0.push_back(to); c0.push_back(co); T0.push_back(To);
        eo += l.n_tot;
        po += n_points[s];
        bo += n_boxes[s];
        ko += (int64_t)l.task_src.size();
        wo += (int64_t)l.items.size();
        mwo += (int64_t)l.mix_items.size();
        to += (int64_t)l.tc_tiles.size();
        co += (int64_t)l.chunk_start.size();
        To += (int64_t)(l.T.size() / T_width);
        if (l.top == 0) m.top = 0;
    }
    m.n_tot = eo;
    auto shift_items = [](const std::vector<WorkItem>& in, int64_t bo_, int64_t ko_, std::vector<WorkItem>& out) {
        for (WorkItem w : in) {
            w.tgt_box += bo_;
            w.task_lo = (int32_t)(w.task_lo + ko_);
            w.task_hi = (int32_t)(w.task_hi + ko_);
            out.push_back(w);
        }
    };
    auto cat_csr = [&](const std::vector<int64_t>& ptr, const std::vector<int64_t>& idx, int64_t slot_off,
                       std::vector<int64_t>& optr, std::vector<int64_t>& oidx) {
        const int64_t base = (int64_t)oidx.size();
        if (optr.empty()) optr.push_back(0);
        for (size_t e = 1; e < ptr.size(); ++e) optr.push_back(base + ptr[e]);
        for (int64_t v : idx) oidx.push_back(v + slot_off * kChunk);
    };
    for (size_t s = 0; s < ls.size(); ++s) {
        const Layout& l = *ls[s];
        for (int64_t v : l.box_off) m.box_off.push_back(v < 0 ? -1 : v + e0[s]);
        m.box_n.insert(m.box_n.end(), l.box_n.begin(), l.box_n.end());
        m.box_nslot.insert(m.box_nslot.end(), l.box_nslot.begin(), l.box_nslot.end());
        m.slot_start.insert(m.slot_start.end(), l.slot_start.begin(), l.slot_start.end());
        m.X.insert(m.X.end(), l.X.begin(), l.X.end());
        for (int64_t v : l.perm_entry) m.perm_entry.push_back(v + e0[s]);
        for (int64_t v : l.perm_point) m.perm_point.push_back(v + p0[s]);
        m.pos.insert(m.pos.end(), l.pos.begin(), l.pos.end());
        m.T.insert(m.T.end(), l.T.begin(), l.T.end());
        for (int64_t v : l.task_src) m.task_src.push_back(v + b0[s]);
        m.task_mask.insert(m.task_mask.end(), l.task_mask.begin(), l.task_mask.end());
        m.task_flags.insert(m.task_flags.end(), l.task_flags.begin(), l.task_flags.end());
        shift_items(l.items, b0[s], k0[s], m.items);
        cat_csr(l.part_ptr, l.part_idx, w0[s], m.part_ptr, m.part_idx);
        shift_items(l.mix_items, b0[s], k0[s], m.mix_items);
        cat_csr(l.tc_part_ptr, l.tc_part_idx, mw0[s], m.tc_part_ptr, m.tc_part_idx);
        for (SrcTile t : l.tc_tiles) {
            t.start += e0[s];
            t.chunk = (int32_t)(t.chunk + c0[s]);
            m.tc_tiles.push_back(t);
        }
        for (TcItem it : l.tc_items) {
            it.row_off += e0[s];
            it.list_lo = (int32_t)(it.list_lo + t0[s]);
            it.list_hi = (int32_t)(it.list_hi + t0[s]);
            m.tc_items.push_back(it);
        }
        for (int64_t v : l.box_chunk0) m.box_chunk0.push_back(v < 0 ? -1 : v + c0[s]);
        for (int64_t v : l.chunk_start) m.chunk_start.push_back(v + e0[s]);
        m.chunk_cnt.insert(m.chunk_cnt.end(), l.chunk_cnt.begin(), l.chunk_cnt.end());
        m.chunk_center.insert(m.chunk_center.end(), l.chunk_center.begin(), l.chunk_center.end());
        m.pairs_direct += l.pairs_direct;
        m.pairs_far += l.pairs_far;
        m.pairs_tc += l.pairs_tc;
    }
    if (m.part_ptr.empty()) m.part_ptr.push_back(0);
    if (m.tc_part_ptr.empty()) m.tc_part_ptr.push_back(0);
    m.tc_n_slots = mwo;
    if (eo > INT32_MAX || to > INT32_MAX || co > INT32_MAX || ko > INT32_MAX)
        throw Error(-1, "merged plan too large (more than 2^31 entries, tasks, tiles or chunks)");
    // up/down boxes grouped by level over all sets
    m.up_level_ptr.assign(Lmax + 2, 0);
    for (int lv = 0; lv <= Lmax; ++lv) {
        m.up_level_ptr[lv] = (int64_t)m.up.size();
        for (size_t s = 0; s < ls.size(); ++s) {
            const Layout& l = *ls[s];
            if (lv + 1 >= (int)l.up_level_ptr.size()) continue;
            for (int64_t i = l.up_level_ptr[lv]; i < l.up_level_ptr[lv + 1]; ++i) {
                UpBox u = l.up[i];
                u.off += e0[s];
                u.dst += e0[s];
                u.T_off += T0[s];
                m.up.push_back(u);
                m.up_leaf.push_back(l.up_leaf[i]);
            }
        }
    }
    m.up_level_ptr[Lmax + 1] = (int64_t)m.up.size();
    // the longest tile lists first over all sets, by length classes as in
    // build_layout (each item writes its own rows, so the order changes no
    // result)
    std::stable_sort(m.tc_items.begin(), m.tc_items.end(), [](const TcItem& a, const TcItem& c) {
        return length_class(a.list_hi - a.list_lo) > length_class(c.list_hi - c.list_lo);
    });
}

}  // namespace skel
