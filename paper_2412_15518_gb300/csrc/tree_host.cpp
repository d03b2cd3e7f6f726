// Host-side octree builder and interaction plan of the GB300 FMM library.
//
// The octree holds one 8x8x8 sub-grid of cells per node (Sec. 4.3.2); the
// GPU kernels walk a fixed stencil of cell offsets instead of interaction
// lists (Sec. 5.5).  This file validates the leaf list, lays the nodes out
// for the device, and builds the stencil lists, the lattice tables of
// leaf-leaf interactions and the work items of the persistent launch.
#include "tree_host.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <unordered_map>
#include <unordered_set>

#include "common.cuh"

namespace otfmm {

namespace {

inline uint64_t nkey(int L, int x, int y, int z) {
    return (uint64_t)L | ((uint64_t)(uint32_t)x << 4) | ((uint64_t)(uint32_t)y << 24) |
           ((uint64_t)(uint32_t)z << 44);
}

}  // namespace

void default_solve_opts(const ot_solve_opts* o, ot_solve_opts& out) {
    out.theta = 0.5;
    out.G = 1.0;
    out.precision = OT_PRECISION_FP64;
    out.am_correction = 1;
    out.self_term = 0;
    out.reserved = 0;
    if (o) out = *o;
}

int check_solve_opts(const ot_solve_opts& o) {
    if (!(o.theta >= 0.3 && o.theta <= 1.0)) return OT_ERR_INVALID_ARG;
    if (o.precision != OT_PRECISION_FP64 && o.precision != OT_PRECISION_FP32_BULK &&
        o.precision != OT_PRECISION_FP32_WIDE)
        return OT_ERR_INVALID_ARG;
    if (!(o.G == o.G)) return OT_ERR_INVALID_ARG;
    return OT_OK;
}

int build_host_tree(const ot_tree_desc& desc, HostTree& t) {
    t = HostTree();
    if (desc.n_leaf <= 0 || !desc.leaves || !(desc.size > 0.0)) return OT_ERR_INVALID_ARG;
    const int n = desc.n_leaf;
    for (int a = 0; a < 3; a++) t.origin[a] = desc.origin[a];
    t.size = desc.size;
    t.n_leaf = n;
    std::unordered_map<uint64_t, int> leafmap;
    std::unordered_set<uint64_t> anc;
    leafmap.reserve(2 * (size_t)n);
    int Lmax = 0;
    for (int i = 0; i < n; i++) {
        const int* l = desc.leaves + 4 * i;
        if (l[0] < 0 || l[0] >= OT_MAX_LEVELS) return OT_ERR_INVALID_TREE;
        for (int a = 1; a < 4; a++)
            if (l[a] < 0 || l[a] >= (1 << l[0])) return OT_ERR_INVALID_TREE;
        if (!leafmap.emplace(nkey(l[0], l[1], l[2], l[3]), i).second) return OT_ERR_INVALID_TREE;
        Lmax = std::max(Lmax, l[0]);
    }
    for (int i = 0; i < n; i++) {
        const int* l = desc.leaves + 4 * i;
        for (int q = l[0] - 1; q >= 0; q--) {
            int s = l[0] - q;
            if (!anc.insert(nkey(q, l[1] >> s, l[2] >> s, l[3] >> s)).second) break;
        }
    }
    // breadth-first layout from the root
    t.leaf_node.assign(n, -1);
    std::vector<std::array<int, 4>> cur{{0, 0, 0, 0}}, next;
    std::vector<std::unordered_map<uint64_t, int>> map;
    int reached = 0;
    for (int L = 0; !cur.empty(); L++) {
        if (L >= OT_MAX_LEVELS) return OT_ERR_INVALID_TREE;
        t.level_first.push_back(t.n_nodes());
        map.emplace_back();
        next.clear();
        for (const auto& nd : cur) {
            uint64_t k = nkey(L, nd[1], nd[2], nd[3]);
            auto lf = leafmap.find(k);
            bool is_leaf = lf != leafmap.end();
            bool is_anc = anc.count(k) != 0;
            if (is_leaf && is_anc) return OT_ERR_INVALID_TREE;   // a leaf inside a leaf
            if (!is_leaf && !is_anc) return OT_ERR_INVALID_TREE; // a hole in the tiling
            int id = t.n_nodes();
            map[L][nkey(L, nd[1], nd[2], nd[3])] = id;
            t.node_level.push_back(L);
            t.node_xyz.insert(t.node_xyz.end(), {nd[1], nd[2], nd[3]});
            t.node_parent.push_back(nd[0]);
            t.node_child.push_back(-1);
            if (is_leaf) {
                t.node_leaf.push_back(lf->second);
                t.leaf_node[lf->second] = id;
                reached++;
            } else {
                t.node_leaf.push_back(-1);
                for (int c = 0; c < 8; c++)
                    next.push_back({id, 2 * nd[1] + (c & 1), 2 * nd[2] + ((c >> 1) & 1),
                                    2 * nd[3] + (c >> 2)});
            }
        }
        cur.swap(next);
    }
    t.node_parent[0] = -1;
    if (reached != n) return OT_ERR_INVALID_TREE;
    t.n_levels = (int)t.level_first.size();
    t.level_first.push_back(t.n_nodes());
    if (t.n_levels - 1 != Lmax) return OT_ERR_INVALID_TREE;
    // first child of each interior node: children were appended in parent order
    for (int v = 1; v < t.n_nodes(); v++) {
        int p = t.node_parent[v];
        if (t.node_child[p] < 0) t.node_child[p] = v;
    }
    // same-level neighbours
    const int N = t.n_nodes();
    t.nbr.assign((size_t)N * 27, -1);
    for (int v = 0; v < N; v++) {
        int L = t.node_level[v], side = 1 << L;
        const int* p = &t.node_xyz[3 * v];
        for (int s = 0; s < 27; s++) {
            int q[3] = {p[0] + s % 3 - 1, p[1] + (s / 3) % 3 - 1, p[2] + s / 9 - 1};
            if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= side || q[1] >= side || q[2] >= side)
                continue;
            auto it = map[L].find(nkey(L, q[0], q[1], q[2]));
            if (it != map[L].end()) t.nbr[(size_t)v * 27 + s] = it->second;
        }
    }
    // 2:1 balance: the region next to a leaf at level L is covered by nodes
    // of level >= L - 1 (the finer side is checked from the finer leaves)
    for (int v = 0; v < N; v++) {
        if (t.node_leaf[v] < 0) continue;
        int L = t.node_level[v], side = 1 << L;
        const int* p = &t.node_xyz[3 * v];
        for (int s = 0; s < 27; s++) {
            if (s == 13 || t.nbr[(size_t)v * 27 + s] >= 0) continue;
            int q[3] = {p[0] + s % 3 - 1, p[1] + (s / 3) % 3 - 1, p[2] + s / 9 - 1};
            if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= side || q[1] >= side || q[2] >= side)
                continue;
            if (L < 1 || map[L - 1].find(nkey(L - 1, q[0] >> 1, q[1] >> 1, q[2] >> 1)) ==
                             map[L - 1].end())
                return OT_ERR_NOT_BALANCED;
        }
    }
    return OT_OK;
}

int build_stencil(const HostTree& t, double theta, HostPlan& p) {
    if (!(theta >= 0.3 && theta <= 1.0)) return OT_ERR_INVALID_ARG;
    p = HostPlan();
    p.theta = theta;
    const double it2 = 1.0 / (theta * theta);
    const int R = (int)std::floor(1.0 / theta + 1e-12);
    const int W = 2 * R + 1;  // children of near parents are at most this far apart
    std::vector<int> near;
    for (int dz = -R; dz <= R; dz++)
        for (int dy = -R; dy <= R; dy++)
            for (int dx = -R; dx <= R; dx++) {
                if (!(dx | dy | dz)) continue;
                if ((double)(dx * dx + dy * dy + dz * dz) <= it2) near.push_back(pack_entry(dx, dy, dz, 1));
            }
    p.n_near = (int)near.size();
    while ((double)(p.near_d2 + 1) <= it2) p.near_d2++;  // the same test as the lists
    auto push = [&](int e) {
        p.entries.push_back(e);
        int d[3] = {entry_dx(e), entry_dy(e), entry_dz(e)};
        double r = std::sqrt((double)(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
        double r3 = r * r * r;
        // D0 and D1 = -R/|R|^3 at R = X_target - X_source = -d (cell units)
        p.tab64.push_back({1.0 / r, d[0] / r3, d[1] / r3, d[2] / r3});
        p.tab32.push_back({(float)(1.0 / r), (float)(d[0] / r3), (float)(d[1] / r3),
                           (float)(d[2] / r3)});
        p.off64.push_back({(double)d[0], (double)d[1], (double)d[2], 0.0});
        p.off32.push_back({(float)d[0], (float)d[1], (float)d[2], 0.0f});
    };
    for (int par = 0; par < 8; par++) {
        int pp[3] = {par & 1, (par >> 1) & 1, par >> 2};
        p.list_first[par] = (int)p.entries.size();
        for (int e : near) push(e);
        for (int dz = -W; dz <= W; dz++)
            for (int dy = -W; dy <= W; dy++)
                for (int dx = -W; dx <= W; dx++) {
                    int d[3] = {dx, dy, dz};
                    if ((double)(dx * dx + dy * dy + dz * dz) <= it2) continue;
                    double P2 = 0.0;
                    for (int a = 0; a < 3; a++) {
                        int D = (pp[a] + d[a]) >> 1;  // floor division: parent offset
                        P2 += (double)D * D;
                    }
                    if (P2 <= it2) push(pack_entry(dx, dy, dz, 0));
                }
        p.list_len[par] = (int)p.entries.size() - p.list_first[par];
    }
    // halo offsets of the parity lists for the lattice kernel
    p.w_far = W;
    p.w_near = R;
    p.hoff_far.assign(p.entries.size(), 0);
    p.hoff_near.assign(p.entries.size(), 0);
    for (int par = 0; par < 8; par++) {
        int pp[3] = {par & 1, (par >> 1) & 1, par >> 2};
        for (int q = 0; q < p.list_len[par]; q++) {
            int e = p.entries[p.list_first[par] + q];
            int d[3] = {entry_dx(e), entry_dy(e), entry_dz(e)};
            p.hoff_far[p.list_first[par] + q] = halo_index(pp[0] + d[0], pp[1] + d[1], pp[2] + d[2], W);
            if (entry_near(e))
                p.hoff_near[p.list_first[par] + q] =
                    halo_index(pp[0] + d[0], pp[1] + d[1], pp[2] + d[2], R);
        }
    }
    // level 0: every non-near pair of the root's 8^3 cells is far
    p.list_first[8] = (int)p.entries.size();
    for (int e : near) push(e);
    for (int dz = -7; dz <= 7; dz++)
        for (int dy = -7; dy <= 7; dy++)
            for (int dx = -7; dx <= 7; dx++) {
                if ((double)(dx * dx + dy * dy + dz * dz) <= it2) continue;
                push(pack_entry(dx, dy, dz, 0));
            }
    p.list_len[8] = (int)p.entries.size() - p.list_first[8];
    p.hoff_far.resize(p.entries.size(), 0);
    p.hoff_near.resize(p.entries.size(), 0);

    // Interaction counts.  For a list and a neighbour slot, count the
    // (target, entry) pairs of that list whose source falls in that slot,
    // split into near and far entries; then every node adds the counts of
    // its existing neighbours by class.
    std::vector<int64_t> cn(kNumLists * 27, 0), cf(kNumLists * 27, 0);
    for (int list = 0; list < kNumLists; list++) {
        for (int c = 0; c < 512; c++) {
            int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
            if (list < 8 && (i & 1) + 2 * (j & 1) + 4 * (k & 1) != list) continue;
            for (int q = 0; q < p.list_len[list]; q++) {
                int e = p.entries[p.list_first[list] + q];
                int s[3] = {i + entry_dx(e), j + entry_dy(e), k + entry_dz(e)};
                int slot = ((s[0] >> 3) + 1) + 3 * ((s[1] >> 3) + 1) + 9 * ((s[2] >> 3) + 1);
                (entry_near(e) ? cn : cf)[list * 27 + slot]++;
            }
        }
    }
    for (int v = 0; v < t.n_nodes(); v++) {
        int L = t.node_level[v];
        bool tl = t.node_leaf[v] >= 0;
        int l0 = L == 0 ? 8 : 0, l1 = L == 0 ? 9 : 8;
        for (int s = 0; s < 27; s++) {
            int nb = t.nbr[(size_t)v * 27 + s];
            if (nb < 0) continue;
            bool sl = t.node_leaf[nb] >= 0;
            for (int list = l0; list < l1; list++) {
                int64_t nn = cn[list * 27 + s], nf = cf[list * 27 + s];
                p.n_m2l += nf;
                if (tl && sl) {
                    p.n_p2p += nn;
                    p.n_lattice += nf;
                    p.n_class[kNearP2P] += nn;
                    p.n_class[kLatticeFar] += nf;
                } else if (tl) {
                    p.n_seam += nn;
                    p.n_class[kM2P] += nn + nf;
                } else if (sl) {
                    p.n_seam += nn;
                    p.n_class[kP2M] += nn + nf;
                } else {
                    p.n_class[kMM] += nf;
                }
            }
        }
    }
    double f[PairClasses][2];
    pair_flops(f);
    for (int c = 0; c < PairClasses; c++) {
        p.flops_am += (double)p.n_class[c] * f[c][1];
        p.flops_noam += (double)p.n_class[c] * f[c][0];
    }
    p.flops_near = (double)p.n_class[kNearP2P] * f[kNearP2P][1];
    double s64[PairClasses], s32[PairClasses];
    pair_flops_split(s64, s32);
    for (int c = 0; c < PairClasses; c++) {
        p.flops_bulk64 += (double)p.n_class[c] * s64[c];
        p.flops_bulk32 += (double)p.n_class[c] * s32[c];
    }
    double fa[PairClasses];
    pair_flops_adjoint(fa);
    for (int c = 0; c < PairClasses; c++) p.flops_adjoint += (double)p.n_class[c] * fa[c];
    double ft[PairClasses];
    pair_flops_tangent(ft);
    for (int c = 0; c < PairClasses; c++) p.flops_tangent += (double)p.n_class[c] * ft[c];
    return OT_OK;
}

namespace {

// Neighbour slots (bit s = slot s of the 27) that the 32 targets of one item
// group (parity par, half) reach through entry e.
uint32_t slot_mask(int par, int half, int e) {
    uint32_t m = 0;
    for (int lane = 0; lane < 32; lane++) {
        const int i = 2 * (lane & 3) + (par & 1);
        const int j = 2 * ((lane >> 2) & 3) + ((par >> 1) & 1);
        const int k = 2 * (2 * half + (lane >> 4)) + (par >> 2);
        const int sx = i + entry_dx(e), sy = j + entry_dy(e), sz = k + entry_dz(e);
        m |= 1u << (((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1));
    }
    return m;
}

// Items of every node that needs the general kernel.  Forward items (kept !=
// null) range over a compacted array of list positions: for each node and
// 32-target group only the entries for which some target has a pair to
// compute (a source exists; a near source of an interior target is a leaf;
// the source of a leaf target is interior) are kept, so whole-warp skips at
// domain boundaries and the descending near pairs of interior cells cost no
// iterations.  With `all` (the adjoint's items), every node gets items over
// its whole list, leaf nodes of level >= 1 without interior neighbours one
// item per parity half (their pairs are all lattice pairs), and an interior
// root items over its own 512 cells as partners (as the forward's).
// For every cell of a node and neighbour slot s, the numbers of far and near
// entries of the cell's parity list whose source lies in slot s:
// out[(c * 27 + s) * 2 + near].
std::vector<int> slot_counts(const HostPlan& p) {
    std::vector<int> cnt((size_t)kCells * 27 * 2, 0);
    for (int c = 0; c < kCells; c++) {
        const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
        const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
        for (int q = 0; q < p.list_len[par]; q++) {
            const int e = p.entries[p.list_first[par] + q];
            const int sx = i + entry_dx(e), sy = j + entry_dy(e), sz = k + entry_dz(e);
            const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
            cnt[((size_t)c * 27 + slot) * 2 + entry_near(e)]++;
        }
    }
    return cnt;
}

// Which pairs of a cell of node v a grouped item walks, by neighbour slot
// (the general kernel's rules): kForward, an interior target pairs with every
// leaf source and with the far interior ones, a leaf target with every
// interior source; kReverse1, the adjoint's pass 1 of an interior cell, its
// leaf partners; kReverse2, its pass 2, the forward rule of an interior
// target.
enum { kForward = 0, kReverse1 = 1, kReverse2 = 2 };

// Groups of node v (level >= 1) for one rule: the pairs of each cell counted
// per neighbour slot, the cells sorted by their counts, 16 groups of 32
// (groups without pairs dropped), each chunked over the list positions; y
// carries pass << 16 (0 for the forward items).
void grouped_items(const HostTree& t, const HostPlan& p, const std::vector<int>& cnt, int v,
                   uint32_t exist, uint32_t leafm, int chunk, int rule, std::vector<Item>& items,
                   std::vector<int64_t>& cost, std::vector<uint16_t>& cells) {
    const int L = t.node_level[v];
    const bool tl = t.node_leaf[v] >= 0;
    int count[kCells];
    for (int c = 0; c < kCells; c++) {
        int n = 0;
        for (int s = 0; s < 27; s++) {
            if (!((exist >> s) & 1)) continue;
            const bool sl = (leafm >> s) & 1;
            const int nf = cnt[((size_t)c * 27 + s) * 2], nn = cnt[((size_t)c * 27 + s) * 2 + 1];
            if (rule == kReverse1) n += sl ? nf + nn : 0;
            else if (tl) n += sl ? 0 : nf + nn;
            else n += sl ? nf + nn : nf;
        }
        count[c] = n;
    }
    int order[kCells];
    for (int c = 0; c < kCells; c++) order[c] = c;
    std::stable_sort(order, order + kCells, [&](int a, int b) { return count[a] > count[b]; });
    int len = 0;
    for (int par = 0; par < 8; par++) len = std::max(len, p.list_len[par]);
    const int step = std::max(1, chunk);
    // pair weights on the scale of the parity-class items' costs
    const int weight = rule == kReverse1 ? 20 : (rule == kReverse2 ? 24 : (tl ? 6 : 9));
    const int pass = rule == kForward ? 0 : rule;
    for (int g = 0; g < kCells / 32; g++) {
        const int mx = count[order[32 * g]];
        if (mx == 0) break;  // sorted: the remaining groups have no pairs either
        const int off = (int)cells.size();
        for (int l = 0; l < 32; l++) cells.push_back((uint16_t)order[32 * g + l]);
        for (int k0 = 0; k0 < len; k0 += step) {
            const int k1 = std::min(len, k0 + step);
            items.push_back({v, L | (g << 8) | (kGroupList << 12) | (pass << 16), k0 | (k1 << 16), off});
            // the busiest lane's pairs in the range, weighted by the pair cost
            cost.push_back((int64_t)mx * (k1 - k0) * weight / len + 1);
        }
    }
}

std::vector<Item> make_items(const HostTree& t, int chunk, const HostPlan& p, bool all,
                             std::vector<int>* lattice_nodes, std::vector<int>* kept,
                             std::vector<Item>* grouped = nullptr,
                             std::vector<uint16_t>* grp_cells = nullptr) {
    std::vector<Item> items;
    std::vector<int64_t> cost;
    std::vector<Item> gitems;
    std::vector<int64_t> gcost;
    std::vector<int> cnt;
    if (grouped || (all && grp_cells)) cnt = slot_counts(p);
    // slot masks per list, parity and half (list 8: the leaf root)
    std::vector<uint32_t> masks[kNumLists][8][2];
    auto masks_of = [&](int list, int par, int half) -> const std::vector<uint32_t>& {
        std::vector<uint32_t>& m = masks[list][par][half];
        if (m.empty())
            for (int q = 0; q < p.list_len[list]; q++)
                m.push_back(slot_mask(par, half, p.entries[p.list_first[list] + q]));
        return m;
    };
    for (int v = 0; v < t.n_nodes(); v++) {
        int L = t.node_level[v];
        bool tl = t.node_leaf[v] >= 0;
        bool seam = false;
        uint32_t exist = 0, leafm = 0;
        for (int s = 0; s < 27; s++) {
            int nb = t.nbr[(size_t)v * 27 + s];
            if (nb < 0) continue;
            exist |= 1u << s;
            if (t.node_leaf[nb] >= 0) leafm |= 1u << s;
            else if (tl) seam = true;
        }
        const uint32_t inner = exist & ~leafm;
        bool lattice_only = tl && L > 0 && !seam;
        if (tl && L > 0 && lattice_nodes) lattice_nodes->push_back(v);
        if (lattice_only && !all) continue;
        const bool root_cells = L == 0 && !tl;  // an interior root: its own cells as sources
        const size_t n_before = items.size();
        if (grouped && L > 0)
            grouped_items(t, p, cnt, v, exist, leafm, chunk, kForward, gitems, gcost, *grp_cells);
        if (all && grp_cells && L > 0 && !tl) {
            // the adjoint: an interior cell's two passes as grouped items
            grouped_items(t, p, cnt, v, exist, leafm, chunk, kReverse1, items, cost, *grp_cells);
            grouped_items(t, p, cnt, v, exist, leafm, chunk, kReverse2, items, cost, *grp_cells);
            continue;
        }
        for (int par = 0; par < 8; par++) {
            int list = root_cells ? kRootList : (L == 0 ? 8 : par);
            int len = root_cells ? kCells : p.list_len[list];
            int step = lattice_only ? len : std::max(1, chunk);
            for (int half = 0; half < 2; half++) {
                int start = 0, n = len;
                if (kept && !root_cells) {
                    const std::vector<uint32_t>& m = masks_of(list, par, half);
                    start = (int)kept->size();
                    for (int q = 0; q < len; q++) {
                        const bool near = entry_near(p.entries[p.list_first[list] + q]) != 0;
                        bool keep;
                        if (tl && L == 0) keep = (m[q] & exist) != 0;  // leaf root: lattice pairs here
                        else if (tl) keep = (m[q] & inner) != 0;
                        else keep = (m[q] & (near ? leafm : exist)) != 0;
                        if (keep) kept->push_back(q);
                    }
                    n = (int)kept->size() - start;
                }
                for (int k0 = 0; k0 < n; k0 += step) {
                    int k1 = std::min(n, k0 + step);
                    items.push_back({v, L | (par << 8) | (half << 11) | (list << 12), start + k0, start + k1});
                    cost.push_back((int64_t)(k1 - k0) * (lattice_only ? 1 : (tl ? 4 : 24)));
                }
            }
        }
        if (grouped && L == 0)
            for (size_t n = n_before; n < items.size(); n++) {
                gitems.push_back(items[n]);
                // the same scale as the grouped items' costs (pairs x weight)
                gcost.push_back(cost[n] * (tl ? 6 : 9) / (tl ? 4 : 24) + 1);
            }
    }
    // longest items first; ties keep the breadth-first node order
    auto by_cost = [](std::vector<Item>& it, const std::vector<int64_t>& c) {
        std::vector<int> order(it.size());
        for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return c[a] > c[b]; });
        std::vector<Item> sorted(it.size());
        for (size_t i = 0; i < order.size(); i++) sorted[i] = it[order[i]];
        return sorted;
    };
    if (grouped) *grouped = by_cost(gitems, gcost);
    return by_cost(items, cost);
}

}  // namespace

void build_items(const HostTree& t, int chunk, HostPlan& p) {
    p.chunk = chunk;
    p.lattice_nodes.clear();
    p.item_entries.clear();
    p.grp_cells.clear();
    p.items = make_items(t, chunk, p, false, &p.lattice_nodes, &p.item_entries, &p.items_grp,
                         &p.grp_cells);
    p.items_adj = make_items(t, chunk, p, true, nullptr, nullptr, nullptr, &p.grp_cells);
}

}  // namespace otfmm
