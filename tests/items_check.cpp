// Host check of the persistent launch's work items (compiled by
// test_items_host.py with the library's host sources): the grouped items of
// the FP64 and FP32-bulk forms (cells of a node regrouped by their pair
// counts, each lane walking its own parity list) must enumerate exactly the
// pairs of the parity-class items (32 cells of one parity class over the
// kept list positions); the adjoint's grouped items of its two passes, and
// its items of an interior root over the root's own cells, must enumerate
// exactly the partners each pass reverses, with every interior target in
// exactly one item that starts its pass-2 range; and every index they
// produce must stay in bounds.
//
// Usage: items_check <leaves.bin> <theta> <chunk>; leaves.bin holds int32
// (L, ix, iy, iz) rows.  Prints "pairs <n> grouped_items <m> bad <b>" and
// exits 1 on any mismatch or out-of-bounds index.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <tuple>
#include <vector>

#include "../paper_2412_15518_gb300/csrc/common.cuh"
#include "../paper_2412_15518_gb300/csrc/tree_host.hpp"

using namespace otfmm;

namespace {
typedef std::tuple<int, int, int, int> Pair;  // node, target cell, entry, kind

// The kernel's pair rules for target cell (i, j, k) of node v and entry e:
// 0 no pair, 1 point masses of a leaf root, 2 leaf source, 3 interior source.
int kind_of(const HostTree& t, int v, int i, int j, int k, int e, int& bad) {
    const int sx = i + entry_dx(e), sy = j + entry_dy(e), sz = k + entry_dz(e);
    const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
    if (sx < -8 || sx >= 16 || sy < -8 || sy >= 16 || sz < -8 || sz >= 16) {
        bad++;
        return 0;
    }
    const int nb = t.nbr[(size_t)v * 27 + slot];
    if (nb < 0) return 0;
    const bool full = t.node_leaf[v] < 0, sleaf = t.node_leaf[nb] >= 0;
    if (!full && sleaf) return t.node_level[v] > 0 ? 0 : 1;
    if (full && !sleaf && entry_near(e)) return 0;
    return sleaf ? 2 : 3;
}
}  // namespace

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    std::vector<int32_t> lv;
    int32_t x;
    while (std::fread(&x, 4, 1, f) == 1) lv.push_back(x);
    std::fclose(f);
    ot_tree_desc d{{0, 0, 0}, 1.0, (int32_t)(lv.size() / 4), lv.data()};
    HostTree t;
    if (build_host_tree(d, t) != OT_OK) return 2;
    HostPlan p;
    if (build_stencil(t, std::atof(argv[2]), p) != OT_OK) return 2;
    build_items(t, std::atoi(argv[3]), p);
    int bad = 0;
    std::multiset<Pair> a, b;
    // parity-class items (kept list positions)
    auto parity_item = [&](const Item& it, std::multiset<Pair>& out) {
        const int v = it.x, par = (it.y >> 8) & 7, half = (it.y >> 11) & 1, list = (it.y >> 12) & 15;
        for (int lane = 0; lane < 32; lane++) {
            const int i = 2 * (lane & 3) + (par & 1), j = 2 * ((lane >> 2) & 3) + ((par >> 1) & 1);
            const int k = 2 * (2 * half + (lane >> 4)) + (par >> 2);
            for (int pos = it.z; pos < it.w; pos++) {
                if (pos < 0 || pos >= (int)p.item_entries.size()) {
                    bad++;
                    continue;
                }
                const int ent = p.list_first[list] + p.item_entries[pos];
                const int kind = kind_of(t, v, i, j, k, p.entries[ent], bad);
                if (kind) out.insert(Pair(v, i + 8 * j + 64 * k, ent, kind));
            }
        }
    };
    for (const Item& it : p.items)
        if (((it.y >> 12) & 15) != kRootList) parity_item(it, a);
    int grouped = 0;
    for (const Item& it : p.items_grp) {
        const int list = (it.y >> 12) & 15;
        if (list == kRootList) continue;
        if (list != kGroupList) {
            if ((it.y & 255) != 0) bad++;  // only level 0 keeps parity-class items
            parity_item(it, b);
            continue;
        }
        grouped++;
        const int v = it.x, k0 = it.z & 0xffff, k1 = it.z >> 16;
        if ((it.y & 255) < 1 || it.w < 0 || (size_t)it.w + 32 > p.grp_cells.size() || k0 >= k1) {
            bad++;
            continue;
        }
        for (int lane = 0; lane < 32; lane++) {
            const int c = p.grp_cells[it.w + lane];
            if (c >= kCells) {
                bad++;
                continue;
            }
            const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
            const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
            const int qend = k1 < p.list_len[par] ? k1 : p.list_len[par];
            for (int q = k0; q < qend; q++) {
                const int ent = p.list_first[par] + q;
                const int kind = kind_of(t, v, i, j, k, p.entries[ent], bad);
                if (kind == 1) bad++;  // leaf roots are level 0
                if (kind) b.insert(Pair(v, c, ent, kind));
            }
        }
    }
    // a cell appears in one group of its node only
    std::set<std::pair<int, int>> seen;
    for (const Item& it : p.items_grp)
        if (((it.y >> 12) & 15) == kGroupList && (it.z & 0xffff) == 0)
            for (int lane = 0; lane < 32; lane++)
                if (!seen.insert({it.x, p.grp_cells[it.w + lane]}).second) bad++;
    if (a != b) bad++;
    // The adjoint's items: interior nodes of level >= 1 as grouped items of
    // pass 1 (leaf partners) and pass 2 (leaf partners and far interior
    // ones) over their cells' whole parity lists; an interior root as items
    // over its own cells (pass 2 with the far ones, |d|^2 > near_d2); every
    // other node keeps parity-class items running both passes.
    std::multiset<Pair> r_want, r_got;
    for (int v = 0; v < t.n_nodes(); v++) {
        if (t.node_level[v] == 0 && t.node_leaf[v] < 0)
            for (int c = 0; c < kCells; c++)
                for (int sc = 0; sc < kCells; sc++) {
                    const int dx = (sc & 7) - (c & 7), dy = ((sc >> 3) & 7) - ((c >> 3) & 7),
                              dz = (sc >> 6) - (c >> 6);
                    if (dx * dx + dy * dy + dz * dz > p.near_d2) r_want.insert(Pair(v, c, -1 - sc, 2));
                }
        if (t.node_level[v] < 1 || t.node_leaf[v] >= 0) continue;
        for (int c = 0; c < kCells; c++) {
            const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
            const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
            for (int q = 0; q < p.list_len[par]; q++) {
                const int ent = p.list_first[par] + q, e = p.entries[ent];
                const int sx = i + entry_dx(e), sy = j + entry_dy(e), sz = k + entry_dz(e);
                const int nb = t.nbr[(size_t)v * 27 + ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1)];
                if (nb < 0) continue;
                const bool pleaf = t.node_leaf[nb] >= 0;
                if (pleaf) r_want.insert(Pair(v, c, ent, 1));
                if (pleaf || !entry_near(e)) r_want.insert(Pair(v, c, ent, 2));
            }
        }
    }
    for (const Item& it : p.items_adj) {
        const int v = it.x, list = (it.y >> 12) & 15;
        if (list == kRootList) {
            // cells [z, w) of the interior root as the partners of the 32
            // cells of one parity class and half
            if (t.node_level[v] != 0 || t.node_leaf[v] >= 0 || it.z < 0 || it.w > kCells || it.z >= it.w) {
                bad++;
                continue;
            }
            const int par = (it.y >> 8) & 7, half = (it.y >> 11) & 1;
            for (int lane = 0; lane < 32; lane++) {
                const int i = 2 * (lane & 3) + (par & 1), j = 2 * ((lane >> 2) & 3) + ((par >> 1) & 1);
                const int k = 2 * (2 * half + (lane >> 4)) + (par >> 2);
                for (int sc = it.z; sc < it.w; sc++) {
                    const int dx = (sc & 7) - i, dy = ((sc >> 3) & 7) - j, dz = (sc >> 6) - k;
                    if (dx * dx + dy * dy + dz * dz > p.near_d2) r_got.insert(Pair(v, i + 8 * j + 64 * k, -1 - sc, 2));
                }
            }
            continue;
        }
        if (list != kGroupList) {
            if (t.node_level[v] == 0 && t.node_leaf[v] < 0) bad++;  // the interior root's items are kRootList
            if (t.node_level[v] >= 1 && t.node_leaf[v] < 0) bad++;  // interior nodes are grouped
            continue;
        }
        const int pass = (it.y >> 16) & 3, k0 = it.z & 0xffff, k1 = it.z >> 16;
        if ((pass != 1 && pass != 2) || t.node_leaf[v] >= 0 || it.w < 0 ||
            (size_t)it.w + 32 > p.grp_cells.size()) {
            bad++;
            continue;
        }
        for (int lane = 0; lane < 32; lane++) {
            const int c = p.grp_cells[it.w + lane];
            if (c >= kCells) {
                bad++;
                continue;
            }
            const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
            const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
            const int qend = k1 < p.list_len[par] ? k1 : p.list_len[par];
            for (int q = k0; q < qend; q++) {
                const int ent = p.list_first[par] + q, e = p.entries[ent];
                const int sx = i + entry_dx(e), sy = j + entry_dy(e), sz = k + entry_dz(e);
                if (sx < -8 || sx >= 16 || sy < -8 || sy >= 16 || sz < -8 || sz >= 16) {
                    bad++;
                    continue;
                }
                const int nb = t.nbr[(size_t)v * 27 + ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1)];
                if (nb < 0) continue;
                const bool pleaf = t.node_leaf[nb] >= 0;
                if (pass == 1 ? pleaf : (pleaf || !entry_near(e))) r_got.insert(Pair(v, c, ent, pass));
            }
        }
    }
    if (r_want != r_got) bad++;
    // The reverse pass forms a target's octupole adjoint from the forward
    // pass's quartic sum once, in the item that starts the target's pass-2
    // range (range start 0): every interior target with a pass-2 partner lies
    // in exactly one such item.
    std::map<std::pair<int, int>, int> first;
    for (const Item& it : p.items_adj) {
        const int list = (it.y >> 12) & 15;
        if (list == kRootList && it.z == 0) {
            const int par = (it.y >> 8) & 7, half = (it.y >> 11) & 1;
            for (int lane = 0; lane < 32; lane++) {
                const int i = 2 * (lane & 3) + (par & 1), j = 2 * ((lane >> 2) & 3) + ((par >> 1) & 1);
                const int k = 2 * (2 * half + (lane >> 4)) + (par >> 2);
                first[{it.x, i + 8 * j + 64 * k}]++;
            }
        } else if (list == kGroupList && ((it.y >> 16) & 3) == 2 && (it.z & 0xffff) == 0) {
            for (int lane = 0; lane < 32; lane++) first[{it.x, (int)p.grp_cells[it.w + lane]}]++;
        }
    }
    std::set<std::pair<int, int>> targets;
    for (const Pair& q : r_want)
        if (std::get<3>(q) == 2) targets.insert({std::get<0>(q), std::get<1>(q)});
    for (const auto& tc : targets)
        if (first.count(tc) == 0 || first[tc] != 1) bad++;
    std::printf("pairs %zu grouped_items %d reverse_pairs %zu bad %d\n", a.size(), grouped, r_want.size(),
                bad);
    return bad ? 1 : 0;
}
