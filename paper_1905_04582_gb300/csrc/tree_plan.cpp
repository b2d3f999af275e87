// Host side of the phylogenetic prior (arXiv:1905.04582, section 2.2): forest
// parsing, message-variance weights, and the cut of each tree into the
// per-CTA parts of tree_prior.cu.  No CUDA calls.
#include "tree_plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

namespace mds {

namespace {

std::string fmt(const char *f, long long a, long long b = 0) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), f, a, b);
    return buf;
}

}  // namespace

std::string parse_forest(int64_t n, int64_t n_nodes, const int64_t *parent, const double *length, ForestShape &f) {
    if (n_nodes < n || n_nodes > 2 * n - 1)
        return fmt("a binary forest over N = %lld tips has N to 2N-1 nodes, got %lld", n, n_nodes);
    f = ForestShape{};
    f.n = n;
    f.n_nodes = n_nodes;
    f.c0.assign(n_nodes, -1);
    f.c1.assign(n_nodes, -1);
    for (int64_t k = 0; k < n_nodes; ++k) {
        const int64_t p = parent[k];
        if (p == -1) continue;
        if (p < n || p >= n_nodes) return fmt("node %lld: parent %lld is not an internal node", k, p);
        if (!(length[k] > 0.0) || !std::isfinite(length[k]))
            return fmt("node %lld: branch length must be finite and > 0", k);
        if (f.c0[p] < 0) f.c0[p] = static_cast<int32_t>(k);
        else if (f.c1[p] < 0) f.c1[p] = static_cast<int32_t>(k);
        else return fmt("node %lld has more than two children", p);
    }
    for (int64_t k = n; k < n_nodes; ++k)
        if (f.c1[k] < 0) return fmt("internal node %lld needs two children", k);
    // heights in post-order from every root (an iterative DFS); a node seen
    // twice or never means a cycle
    f.height.assign(n_nodes, -1);
    for (int64_t r = 0; r < n_nodes; ++r) {
        if (parent[r] != -1) continue;
        if (r < n) {
            f.lone.push_back(static_cast<int32_t>(r));
            f.height[r] = 0;
            continue;
        }
        f.roots.push_back(static_cast<int32_t>(r));
        std::vector<std::pair<int32_t, int>> st{{static_cast<int32_t>(r), 0}};
        while (!st.empty()) {
            auto &top = st.back();
            const int32_t u = top.first;
            if (u < n) {
                f.height[u] = 0;
                st.pop_back();
                continue;
            }
            if (top.second < 2) {
                const int32_t ch = top.second == 0 ? f.c0[u] : f.c1[u];
                top.second++;
                if (f.height[ch] != -1 || static_cast<int64_t>(st.size()) > n_nodes)
                    return "the parent links do not form a forest";
                st.push_back({ch, 0});
                continue;
            }
            f.height[u] = 1 + std::max(f.height[f.c0[u]], f.height[f.c1[u]]);
            f.order.push_back(u);
            st.pop_back();
        }
    }
    for (int64_t k = 0; k < n_nodes; ++k)
        if (f.height[k] < 0) return fmt("node %lld is not connected to a root", k);
    return "";
}

void tree_weights(const ForestShape &f, const double *length, double tau0, double tau_u, int d,
                  std::vector<TreeWeights> &wt, std::vector<double> &root_cinv, double &cst) {
    const int64_t n = f.n;
    const double log2pi = 1.8378770664093454836;
    const double hd = 0.5 * d;
    std::vector<double> up_v(f.n_nodes, 0.0), dn_v(f.n_nodes, 0.0);
    wt.assign(f.n_nodes, TreeWeights{});
    root_cinv.clear();
    cst = 0.0;
    // upward variances: children before parents
    for (int32_t k : f.order) {
        const int32_t a = f.c0[k], b = f.c1[k];
        const double va = up_v[a] + length[a], vb = up_v[b] + length[b], sv = va + vb;
        wt[k].alpha = vb / sv;
        wt[k].cinv = 1.0 / sv;
        up_v[k] = va * vb / sv;
        cst -= hd * (log2pi + std::log(sv));
    }
    for (int32_t r : f.roots) {
        const double sv = up_v[r] + tau0;
        root_cinv.push_back(1.0 / sv);
        cst -= hd * (log2pi + std::log(sv));
        dn_v[r] = tau0;
    }
    cst -= hd * (log2pi + std::log(tau_u)) * static_cast<double>(f.lone.size());
    // downward variances: parents before children
    for (auto it = f.order.rbegin(); it != f.order.rend(); ++it) {
        const int32_t k = *it;
        const double vk = dn_v[k];
        for (int side = 0; side < 2; ++side) {
            const int32_t ch = side == 0 ? f.c0[k] : f.c1[k], sib = side == 0 ? f.c1[k] : f.c0[k];
            const double vs = up_v[sib] + length[sib];
            const double beta = vs / (vk + vs);
            const double vc = vk * vs / (vk + vs) + length[ch];
            const double g = ch < n ? 1.0 / vc : 0.0;
            if (side == 0) {
                wt[k].beta0 = beta;
                wt[k].g0 = g;
            } else {
                wt[k].beta1 = beta;
                wt[k].g1 = g;
            }
            if (ch >= n) dn_v[ch] = vc;
        }
    }
}

void plan_forest(const ForestShape &f, const std::vector<TreeWeights> &wt, int d, TreePlan &p) {
    const int64_t n = f.n;
    const auto &c0 = f.c0, &c1 = f.c1, &height = f.height;
    p = TreePlan{};
    std::vector<int32_t> sz(f.n_nodes, 0);  // internal nodes of each subtree
    for (int32_t k : f.order) sz[k] = 1 + (c0[k] >= n ? sz[c0[k]] : 0) + (c1[k] >= n ? sz[c1[k]] : 0);
    int32_t m_max = 0;
    for (int32_t r : f.roots) m_max = std::max(m_max, sz[r]);
    const int ncl = std::max(1, std::min(kTreeMaxCluster, (m_max + 63) / 64));
    p.cluster = ncl;
    p.parts.assign(f.roots.size() * ncl, TreePart{});
    p.node_off.push_back(0);
    p.tip_off.push_back(0);
    std::vector<int32_t> local(f.n_nodes, -1), slot_of(f.n_nodes, -1);
    std::vector<char> is_top(f.n_nodes, 0);
    auto by_height = [&](int32_t a, int32_t b) { return height[a] < height[b] || (height[a] == height[b] && a < b); };
    for (size_t t = 0; t < f.roots.size(); ++t) {
        const int32_t r = f.roots[t];
        const int32_t S = std::max<int32_t>(1, (sz[r] + 4 * ncl - 1) / (4 * ncl));
        // the cut: from the root, a node whose subtree holds at most S
        // internal nodes is a block root, any other one a top node
        std::vector<int32_t> top, blocks;
        {
            std::vector<int32_t> st{r};
            while (!st.empty()) {
                const int32_t u = st.back();
                st.pop_back();
                if (sz[u] <= S) {
                    blocks.push_back(u);
                    continue;
                }
                top.push_back(u);
                is_top[u] = 1;
                if (c1[u] >= n) st.push_back(c1[u]);
                if (c0[u] >= n) st.push_back(c0[u]);
            }
        }
        std::sort(blocks.begin(), blocks.end(),
                  [&](int32_t a, int32_t b) { return sz[a] > sz[b] || (sz[a] == sz[b] && a < b); });
        std::vector<int64_t> load(ncl, 0);
        load[0] = 2 * static_cast<int64_t>(top.size());
        std::vector<std::vector<int32_t>> owned(ncl);
        for (size_t q = 0; q < blocks.size(); ++q) {
            slot_of[blocks[q]] = static_cast<int32_t>(q);
            const int cbest = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
            owned[cbest].push_back(blocks[q]);
            load[cbest] += sz[blocks[q]];
        }
        const int32_t n_slots = static_cast<int32_t>(blocks.size());
        std::sort(top.begin(), top.end(), by_height);
        for (int cr = 0; cr < ncl; ++cr) {
            TreePart &pt = p.parts[t * ncl + cr];
            // the part's block nodes: the whole subtrees of its block roots
            std::vector<int32_t> bn;
            for (int32_t b : owned[cr]) {
                std::vector<int32_t> st{b};
                while (!st.empty()) {
                    const int32_t u = st.back();
                    st.pop_back();
                    bn.push_back(u);
                    if (c0[u] >= n) st.push_back(c0[u]);
                    if (c1[u] >= n) st.push_back(c1[u]);
                }
            }
            std::sort(bn.begin(), bn.end(), by_height);
            pt.m_blk = static_cast<int32_t>(bn.size());
            pt.n_prox = cr == 0 ? n_slots : 0;
            pt.m_top = cr == 0 ? static_cast<int32_t>(top.size()) : 0;
            for (size_t q = 0; q < bn.size(); ++q) local[bn[q]] = static_cast<int32_t>(q);
            const int32_t top0 = pt.m_blk + pt.n_prox;
            if (cr == 0)
                for (size_t q = 0; q < top.size(); ++q) local[top[q]] = top0 + static_cast<int32_t>(q);
            const int32_t tip0 = static_cast<int32_t>(p.tip_items.size());
            auto record = [&](int32_t k) {
                TreeNode rc{};
                int32_t ref[2];
                for (int side = 0; side < 2; ++side) {
                    const int32_t ch = side == 0 ? c0[k] : c1[k];
                    if (ch < n) {
                        ref[side] = -(static_cast<int32_t>(p.tip_items.size()) - tip0 + 1);
                        p.tip_items.push_back(ch);
                    } else if (is_top[k] && !is_top[ch]) {
                        ref[side] = pt.m_blk + slot_of[ch];  // a block root: its proxy
                    } else {
                        ref[side] = local[ch];
                    }
                }
                rc.c0 = ref[0];
                rc.c1 = ref[1];
                rc.alpha = wt[k].alpha;
                rc.cinv = wt[k].cinv;
                rc.beta0 = wt[k].beta0;
                rc.beta1 = wt[k].beta1;
                rc.g0 = wt[k].g0;
                rc.g1 = wt[k].g1;
                p.nodes.push_back(rc);
                p.node_id.push_back(k);
            };
            // level bounds of `mem` (sorted by height, local indices from
            // `base`); `small`: the first of the last run of levels with at
            // most 32 nodes each (warp 0's work)
            auto levels = [&](const std::vector<int32_t> &mem, int32_t base, int32_t &nlv, int32_t &small) {
                const int32_t l0 = static_cast<int32_t>(p.lv_start.size());
                int prev = -1;
                for (size_t q = 0; q < mem.size(); ++q) {
                    if (height[mem[q]] != prev) {
                        p.lv_start.push_back(base + static_cast<int32_t>(q));
                        prev = height[mem[q]];
                    }
                }
                nlv = static_cast<int32_t>(p.lv_start.size()) - l0;
                small = nlv;
                while (small > 0) {
                    const int32_t a0 = p.lv_start[l0 + small - 1];
                    const int32_t a1 = small < nlv ? p.lv_start[l0 + small] : base + static_cast<int32_t>(mem.size());
                    if (a1 - a0 > 32) break;
                    --small;
                }
            };
            pt.lv0 = static_cast<int32_t>(p.lv_start.size());
            for (int32_t k : bn) record(k);
            levels(bn, 0, pt.nlv_blk, pt.small_blk);
            if (cr == 0) {
                for (int32_t q = 0; q < n_slots; ++q) {  // proxies: no work of their own
                    p.nodes.push_back(TreeNode{});
                    p.node_id.push_back(-1);
                }
                for (int32_t k : top) record(k);
                levels(top, top0, pt.nlv_top, pt.small_top);
                pt.root_loc = is_top[r] ? local[r] : pt.m_blk + slot_of[r];
            } else {
                pt.nlv_top = pt.small_top = 0;
                pt.root_loc = -1;
            }
            pt.exp0 = static_cast<int32_t>(p.exp_loc.size());
            for (int32_t b : owned[cr]) {
                p.exp_loc.push_back(local[b]);
                p.exp_slot.push_back(slot_of[b]);
            }
            pt.exp1 = static_cast<int32_t>(p.exp_loc.size());
            pt.n_slots = n_slots;
            pt.xch_off = p.xch_total;
            p.node_off.push_back(static_cast<int32_t>(p.nodes.size()));
            p.tip_off.push_back(static_cast<int32_t>(p.tip_items.size()));
            // records, up / down means of the part's nodes, tip locations, tip
            // downward means and gradient scales, level bounds
            const int64_t m = p.node_off.back() - p.node_off[p.node_off.size() - 2];
            const int64_t kt = static_cast<int64_t>(p.tip_items.size()) - tip0;
            const int64_t fp = m * static_cast<int64_t>(sizeof(TreeNode)) + ((2 * m + 2 * kt) * d + kt) * 8 +
                               4 * static_cast<int64_t>(pt.nlv_blk + pt.nlv_top);
            p.max_fp = std::max(p.max_fp, fp);
            pt.scr_off = p.scr_total;
            p.scr_total += (2 * m + 2 * kt) * d + kt;
        }
        p.xch_total += 2 * static_cast<int64_t>(n_slots) * d;
    }
}

std::string check_plan(const ForestShape &f, const TreePlan &p, int d) {
    const int64_t n = f.n;
    const int ncl = p.cluster;
    if (ncl < 1 || ncl > kTreeMaxCluster) return "cluster size out of range";
    if (p.parts.size() != f.roots.size() * ncl || p.node_off.size() != p.parts.size() + 1 ||
        p.tip_off.size() != p.parts.size() + 1 || p.node_id.size() != p.nodes.size())
        return "array sizes";
    // the tree of every node (roots in id order)
    std::vector<int32_t> tree_of(f.n_nodes, -1), parent(f.n_nodes, -1);
    for (int32_t k = static_cast<int32_t>(n); k < f.n_nodes; ++k) {
        parent[f.c0[k]] = k;
        parent[f.c1[k]] = k;
    }
    for (size_t t = 0; t < f.roots.size(); ++t) tree_of[f.roots[t]] = static_cast<int32_t>(t);
    for (auto it = f.order.rbegin(); it != f.order.rend(); ++it)
        if (tree_of[*it] < 0) tree_of[*it] = tree_of[parent[*it]];
    for (int32_t k = 0; k < n; ++k)
        if (parent[k] >= 0) tree_of[k] = tree_of[parent[k]];
    std::vector<int> seen(f.n_nodes, 0);
    int64_t xch_end = 0;
    for (size_t t = 0; t < f.roots.size(); ++t) {
        const TreePart &p0 = p.parts[t * ncl];
        const int32_t n_slots = p0.n_slots;
        if (p0.xch_off < xch_end || p0.xch_off + 2LL * n_slots * d > p.xch_total) return fmt("tree %lld: exchange", t);
        xch_end = p0.xch_off + 2LL * n_slots * d;
        std::vector<int32_t> slot_root(n_slots, -1);
        std::vector<int> exported(n_slots, 0);
        for (int cr = 0; cr < ncl; ++cr) {
            const size_t pi = t * ncl + cr;
            const TreePart &pt = p.parts[pi];
            const int32_t nb = p.node_off[pi], m = p.node_off[pi + 1] - nb;
            const int32_t tb = p.tip_off[pi], k = p.tip_off[pi + 1] - tb;
            if (m < 0 || k < 0) return fmt("part %lld: offsets", pi);
            if (pt.n_slots != n_slots || pt.xch_off != p0.xch_off) return fmt("part %lld: exchange", pi);
            if (cr > 0 && (pt.n_prox != 0 || pt.m_top != 0 || pt.nlv_top != 0 || pt.root_loc != -1))
                return fmt("part %lld: a top outside CTA 0", pi);
            if (cr == 0 && pt.n_prox != n_slots) return fmt("part %lld: proxies", pi);
            if (pt.m_blk + pt.n_prox + pt.m_top != m) return fmt("part %lld: node counts", pi);
            const int32_t top0 = pt.m_blk + pt.n_prox;
            // levels of each run: increasing starts, one height per level,
            // increasing heights, narrow from `small` on
            std::vector<int32_t> level_of(m, -1);
            auto check_levels = [&](int32_t l0, int32_t nlv, int32_t small, int32_t lo, int32_t hi) -> std::string {
                if (nlv < 0 || small < 0 || small > nlv || (nlv == 0 && hi > lo)) return "level count";
                if (nlv > 0 && p.lv_start[l0] != lo) return "first level";
                int prev_h = -1;
                for (int32_t l = 0; l < nlv; ++l) {
                    const int32_t a = p.lv_start[l0 + l], b = l + 1 < nlv ? p.lv_start[l0 + l + 1] : hi;
                    if (a >= b || a < lo || b > hi) return "level bounds";
                    if (l >= small && b - a > 32) return "a wide level in the warp run";
                    const int h = f.height[p.node_id[nb + a]];
                    if (h <= prev_h) return "level heights";
                    prev_h = h;
                    for (int32_t i = a; i < b; ++i) {
                        if (f.height[p.node_id[nb + i]] != h) return "mixed heights in a level";
                        level_of[i] = l;
                    }
                }
                return "";
            };
            if (pt.lv0 < 0 || pt.lv0 + pt.nlv_blk + pt.nlv_top > static_cast<int32_t>(p.lv_start.size()))
                return fmt("part %lld: level range", pi);
            std::string e = check_levels(pt.lv0, pt.nlv_blk, pt.small_blk, 0, pt.m_blk);
            if (e.empty()) e = check_levels(pt.lv0 + pt.nlv_blk, pt.nlv_top, pt.small_top, top0, m);
            if (!e.empty()) return fmt("part %lld: ", pi) + e;
            // records: each node once, in its tree; children as the forest has them
            std::vector<int> tip_seen(k, 0);
            for (int32_t i = 0; i < m; ++i) {
                const int32_t id = p.node_id[nb + i];
                const bool proxy = i >= pt.m_blk && i < top0;
                if (proxy) {
                    if (id != -1) return fmt("part %lld: proxy %lld carries a node", pi, i);
                    continue;
                }
                if (id < n || id >= f.n_nodes || tree_of[id] != static_cast<int32_t>(t))
                    return fmt("part %lld: record %lld is not an internal node of the tree", pi, i);
                if (seen[id]++) return fmt("node %lld in two parts", id);
                const bool top = i >= top0;
                const TreeNode &rc = p.nodes[nb + i];
                const int32_t ref[2] = {rc.c0, rc.c1}, ch[2] = {f.c0[id], f.c1[id]};
                for (int s = 0; s < 2; ++s) {
                    if (ref[s] < 0) {
                        const int32_t ti = -ref[s] - 1;
                        if (ti >= k || p.tip_items[tb + ti] != ch[s]) return fmt("node %lld: tip child", id);
                        if (tip_seen[ti]++) return fmt("node %lld: tip referenced twice", id);
                    } else if (top && ref[s] >= pt.m_blk && ref[s] < top0) {
                        const int32_t slot = ref[s] - pt.m_blk;
                        if (ch[s] < n || slot_root[slot] != -1) return fmt("node %lld: proxy child", id);
                        slot_root[slot] = ch[s];
                    } else {
                        if (ref[s] >= m || p.node_id[nb + ref[s]] != ch[s]) return fmt("node %lld: child", id);
                        if ((ref[s] >= top0) != top) return fmt("node %lld: child across the cut", id);
                        if (level_of[ref[s]] < 0 || level_of[ref[s]] >= level_of[i])
                            return fmt("node %lld: child not below", id);
                    }
                }
            }
            for (int32_t i = 0; i < k; ++i) {
                if (!tip_seen[i]) return fmt("part %lld: tip %lld unreferenced", pi, i);
                const int32_t tip = p.tip_items[tb + i];
                if (tip < 0 || tip >= n || tree_of[tip] != static_cast<int32_t>(t) || seen[tip]++)
                    return fmt("part %lld: tip %lld", pi, i);
            }
            // exports: block roots of this part
            if (pt.exp0 < 0 || pt.exp1 < pt.exp0 || pt.exp1 > static_cast<int32_t>(p.exp_loc.size()))
                return fmt("part %lld: export range", pi);
            for (int32_t e2 = pt.exp0; e2 < pt.exp1; ++e2) {
                const int32_t loc = p.exp_loc[e2], slot = p.exp_slot[e2];
                if (loc < 0 || loc >= pt.m_blk || slot < 0 || slot >= n_slots || exported[slot]++)
                    return fmt("part %lld: export %lld", pi, e2);
            }
            if (pt.scr_off < 0 || pt.scr_off + (2LL * m + 2LL * k) * d + k > p.scr_total)
                return fmt("part %lld: scratch", pi);
            const int64_t fp = static_cast<int64_t>(m) * static_cast<int64_t>(sizeof(TreeNode)) +
                               ((2LL * m + 2LL * k) * d + k) * 8 + 4LL * (pt.nlv_blk + pt.nlv_top);
            if (fp > p.max_fp) return fmt("part %lld: footprint", pi);
        }
        for (int32_t s = 0; s < n_slots; ++s)
            if (!exported[s]) return fmt("tree %lld: slot %lld not exported", t, s);
        // each proxy stands for the block root exported in its slot
        for (int cr = 0; cr < ncl; ++cr) {
            const size_t pi = t * ncl + cr;
            const TreePart &pt = p.parts[pi];
            for (int32_t e2 = pt.exp0; e2 < pt.exp1; ++e2) {
                const int32_t id = p.node_id[p.node_off[pi] + p.exp_loc[e2]];
                const int32_t slot = p.exp_slot[e2];
                if (id == f.roots[t]) {
                    if (p0.root_loc != p0.m_blk + slot) return fmt("tree %lld: root proxy", t);
                } else if (slot_root[slot] != id) {
                    return fmt("tree %lld: proxy of slot %lld", t, slot);
                }
            }
        }
        if (p0.root_loc < 0 || p0.root_loc >= p.node_off[t * ncl + 1] - p.node_off[t * ncl])
            return fmt("tree %lld: root", t);
        if (p0.root_loc >= p0.m_blk + p0.n_prox && p.node_id[p.node_off[t * ncl] + p0.root_loc] != f.roots[t])
            return fmt("tree %lld: root record", t);
    }
    for (int32_t k = 0; k < f.n_nodes; ++k) {
        const bool in_tree = tree_of[k] >= 0;
        if (in_tree && seen[k] != 1) return fmt("node %lld covered %lld times", k, seen[k]);
    }
    return "";
}

}  // namespace mds
