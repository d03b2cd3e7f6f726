// Host-side octree builder and interaction plan of the GB300 FMM library.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/octofmm.h"

namespace otfmm {

struct HostTree {
    int n_levels = 0;  // Lmax + 1
    int n_leaf = 0;
    double origin[3] = {0, 0, 0};
    double size = 1.0;
    // nodes in breadth-first order, children of a node contiguous in octant
    // order (bit 0 = x, bit 1 = y, bit 2 = z)
    std::vector<int> level_first;  // [n_levels + 1]
    std::vector<int> node_level, node_leaf, node_parent, node_child;
    std::vector<int> node_xyz;     // [n_nodes][3]
    std::vector<int> nbr;          // [n_nodes][27], slot = (ox+1) + 3 (oy+1) + 9 (oz+1)
    std::vector<int> leaf_node;    // [n_leaf] node index of each caller leaf
    int n_nodes() const { return (int)node_level.size(); }
    // leaf and interior nodes of level L (0 outside the tree)
    int leaf_nodes_at(int L) const {
        if (L < 0 || L >= n_levels) return 0;
        int n = 0;
        for (int v = level_first[L]; v < level_first[L + 1]; v++) n += node_leaf[v] >= 0;
        return n;
    }
    int interior_nodes_at(int L) const {
        if (L < 0 || L >= n_levels) return 0;
        return level_first[L + 1] - level_first[L] - leaf_nodes_at(L);
    }
    // Which of the two upward (M2M) kernels level L needs: bit 0 cells with
    // interior children, bit 1 cells with leaf children.
    int m2m_kinds(int L) const {
        return (interior_nodes_at(L + 1) > 0 ? 1 : 0) | (leaf_nodes_at(L + 1) > 0 ? 2 : 0);
    }
    // Which of the two downward (L2L) kernels level L needs: bit 0 the
    // level's own interior nodes below the root (an interior root has no
    // parent expansion to add) or a root leaf, bit 1 its leaf children.
    int l2l_kinds(int L) const {
        const bool own = L == 0 ? leaf_nodes_at(0) > 0 : interior_nodes_at(L) > 0;
        return (own ? 1 : 0) | (leaf_nodes_at(L + 1) > 0 ? 2 : 0);
    }
};

// Solve options: the defaults (theta 0.5, G 1, FP64, correction on, no
// self term) or a copy of *o; and their check (theta in [0.3, 1], a known
// precision form, G not NaN), shared by every solve entry point.
void default_solve_opts(const ot_solve_opts* o, ot_solve_opts& out);
int check_solve_opts(const ot_solve_opts& o);

// Builds the tree; returns OT_OK, OT_ERR_INVALID_ARG, OT_ERR_INVALID_TREE or
// OT_ERR_NOT_BALANCED.
int build_host_tree(const ot_tree_desc& desc, HostTree& t);

struct Tab4d { double x, y, z, w; };
struct Tab4f { float x, y, z, w; };
struct Item { int x, y, z, w; };

constexpr int kNumLists = 9;  // 8 parity classes at L >= 1, one list at L = 0

// Pair classes: lattice far (two leaf cells), exact near (two leaf cells),
// multipole source on a leaf target, leaf source on an interior target, two
// interior cells.
enum { kLatticeFar = 0, kNearP2P = 1, kM2P = 2, kP2M = 3, kMM = 4, PairClasses = 5 };

// Flops of one pair of each class, [class][am] (counted from the executed
// formula; fma = 2).
void pair_flops(double out[PairClasses][2]);
// FP64 and FP32 flops of one pair of each class in the FP32-bulk form (the
// split pair, with the correction).
void pair_flops_split(double f64[PairClasses], double f32[PairClasses]);
// FP64 flops of the reverse of one pair of each class in the adjoint's
// interaction sweep (with the correction).
void pair_flops_adjoint(double out[PairClasses]);
// FP64 flops of one pair of each class in the tangent solve (dual numbers:
// value and tangent, with the correction).
void pair_flops_tangent(double out[PairClasses]);

// Stencil and work list of a tree for one opening parameter.
struct HostPlan {
    double theta = 0.0;
    int chunk = 0;                    // stencil entries per item of an interior target
    std::vector<int> entries;         // packed offsets (see pack_entry)
    std::vector<Tab4d> tab64;         // (1/|d|, d/|d|^3) per entry, cell units
    std::vector<Tab4f> tab32;
    std::vector<Tab4d> off64;         // (dx, dy, dz, 0) per entry
    std::vector<Tab4f> off32;
    int list_first[kNumLists] = {0};
    int list_len[kNumLists] = {0};
    int n_near = 0;                   // near offsets (first entries of every list)
    int near_d2 = 0;                  // largest integer |d|^2 classified near
    int w_far = 0, w_near = 0;        // halo widths of the lattice kernel
    std::vector<int> hoff_far, hoff_near;  // halo offsets per entry (parity lists)
    std::vector<int> lattice_nodes;   // leaf nodes of level >= 1
    std::vector<Item> items;          // ranges over item_entries (kRootList: over root cells)
    std::vector<int> item_entries;    // list positions kept per node and target group
    std::vector<Item> items_adj;      // every node, ranges over the lists themselves
    std::vector<Item> items_grp;      // the forward items with the nodes of level >= 1
                                      // as grouped items (kGroupList)
    std::vector<uint16_t> grp_cells;  // 32 node-local cells per group
    int64_t n_m2l = 0, n_p2p = 0, n_seam = 0, n_lattice = 0;
    int64_t n_class[PairClasses] = {0, 0, 0, 0, 0};
    double flops_am = 0.0, flops_noam = 0.0;  // one interaction launch
    double flops_near = 0.0;                  // the part kept in FP64 by the wide FP32 form
    double flops_bulk64 = 0.0, flops_bulk32 = 0.0;  // FP32-bulk form, with the correction
    double flops_adjoint = 0.0;                     // reverse sweep of the interactions
    double flops_tangent = 0.0;                     // tangent solve's interactions
};

// Stencil lists for theta (0.3 <= theta <= 1) and the interaction counts of
// the tree; no work items.
int build_stencil(const HostTree& t, double theta, HostPlan& p);

// Work items of the persistent launch for a given chunk length: interior
// targets (chunked; an interior root's items range over its 512 cells as
// sources), leaf targets that border interior cells (their pairs with
// interior cells), and a leaf root; the leaf-leaf pairs of leaf nodes of
// level >= 1 go to the lattice kernel (lattice_nodes).  The adjoint's items
// (items_adj) cover every node and use the stencil lists at every level.
// items_grp holds the same work with the targets of each node of level >= 1
// regrouped: its 512 cells sorted by their number of pairs and taken 32 at a
// time (grp_cells), so that the lanes of a warp have nearly equal work.
void build_items(const HostTree& t, int chunk, HostPlan& p);

}  // namespace otfmm
