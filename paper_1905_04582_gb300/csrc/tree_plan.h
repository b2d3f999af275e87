// Host side of the phylogenetic prior (arXiv:1905.04582, section 2.2): the
// forest's shape, the message variances folded into per-node weights, and
// the cut of each tree into per-CTA parts that tree_prior.cu evaluates.
// Host-only code (no CUDA calls), shared by mds_set_tree_prior and the plan
// check of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "mds_internal.h"

namespace mds {

struct ForestShape {
    int64_t n = 0, n_nodes = 0;          // tips 0..n-1, internal nodes n..n_nodes-1
    std::vector<int32_t> c0, c1;         // children of internal nodes (-1 for tips)
    std::vector<int32_t> height;         // 0 at tips, 1 + the children's largest above
    std::vector<int32_t> order;          // internal nodes, children before parents
    std::vector<int32_t> roots;          // roots that are internal nodes, in id order
    std::vector<int32_t> lone;           // tips that are roots (unsequenced items)
};

// Checks that parent[] (-1 for roots) and length[] (> 0 for non-roots)
// describe a binary forest over the n tips; fills `f`.  Returns "" or the
// reason it is not one.
std::string parse_forest(int64_t n, int64_t n_nodes, const int64_t *parent, const double *length, ForestShape &f);

struct TreeWeights {
    double alpha = 0, cinv = 0, beta0 = 0, beta1 = 0, g0 = 0, g1 = 0;  // as in TreeNode
};

// Message variances (they depend on the tree alone) folded into per-node
// weights; root_cinv[t] = 1 / (v_root + tau0) per tree; `cst` receives the
// 2 pi and branch-variance log-determinant terms of the density (the
// -N/2 log|Sigma| term is the caller's).
void tree_weights(const ForestShape &f, const double *length, double tau0, double tau_u, int d,
                  std::vector<TreeWeights> &wt, std::vector<double> &root_cinv, double &cst);

// The per-CTA schedules of TreeArgs, host copies.
struct TreePlan {
    int cluster = 1;
    std::vector<TreeNode> nodes;
    std::vector<int32_t> node_id;        // per record: the forest node, -1 for a proxy
    std::vector<TreePart> parts;
    std::vector<int32_t> node_off, tip_items, tip_off, lv_start, exp_loc, exp_slot;
    int64_t max_fp = 0;                  // bytes of the largest part's records and messages
    int64_t scr_total = 0;               // doubles of all parts' messages (global scratch)
    int64_t xch_total = 0;               // doubles of all exchange arrays
};

// Cuts every tree into blocks (the largest subtrees of at most S internal
// nodes, S = ceil(m / (4 C))) and a top, assigns the blocks to the C CTAs
// of the tree's cluster (longest first to the least loaded; CTA 0 starts
// with twice the top's size), and lays out each part's records and levels.
void plan_forest(const ForestShape &f, const std::vector<TreeWeights> &wt, int d, TreePlan &p);

// Checks the plan against the forest: every internal node and tip in
// exactly one part, child references and levels consistent, exports and
// proxies matched, offsets in bounds.  Returns "" or the first violation.
std::string check_plan(const ForestShape &f, const TreePlan &p, int d);

}  // namespace mds
