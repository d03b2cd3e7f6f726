// Pins the compile-time near stencil of the lattice kernel (theta = 0.5)
// against the plan built on the host: the 16 representatives and their
// negatives are exactly the offsets 0 < |d|^2 <= 4 of the plan's near lists,
// the constant factors are 1/|d| and 1/|d|^3 to within an ulp, and the
// kernel's halo offsets of d and -d are the plan's for every parity class.
// Prints the number of failed checks.
#include <cmath>
#include <cstdio>
#include <set>
#include <tuple>
#include <vector>

#include "../paper_2412_15518_gb300/csrc/lattice.hpp"
#include "../paper_2412_15518_gb300/csrc/tree_host.hpp"

using namespace otfmm;

static bool within_ulp(double a, double b) {
    return std::fabs(a - b) <= std::nextafter(std::fabs(b), INFINITY) - std::fabs(b);
}

int main() {
    int bad = 0;
    // the stencil's offsets
    std::set<std::tuple<int, int, int>> stencil;
    for (int n = 0; n < 16; n++) {
        const int c = near2_code(n);
        const int dx = c % 5 - 2, dy = (c / 5) % 5 - 2, dz = c / 25 - 2;
        const int r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < 1 || r2 > 4) bad++;
        stencil.insert({dx, dy, dz});
        stencil.insert({-dx, -dy, -dz});
        if (!within_ulp(near2_inv_r(r2), 1.0 / std::sqrt((double)r2))) bad++;
        if (!within_ulp(near2_inv_r3(r2), 1.0 / (r2 * std::sqrt((double)r2)))) bad++;
    }
    // the plan of a level-1 tree at theta = 0.5
    std::vector<int> leaves;
    for (int k = 0; k < 2; k++)
        for (int j = 0; j < 2; j++)
            for (int i = 0; i < 2; i++) leaves.insert(leaves.end(), {1, i, j, k});
    ot_tree_desc desc = {};
    desc.size = 1.0;
    desc.n_leaf = 8;
    desc.leaves = leaves.data();
    HostTree t;
    HostPlan p;
    if (build_host_tree(desc, t) != OT_OK || build_stencil(t, 0.5, p) != OT_OK) {
        std::printf("plan failed\n1\n");
        return 1;
    }
    if (p.n_near != 32 || p.w_near != 2) bad++;  // the kernel's dispatch condition
    for (int par = 0; par < 8; par++) {
        const int px = par & 1, py = (par >> 1) & 1, pz = par >> 2;
        std::set<std::tuple<int, int, int>> listed;
        std::set<int> hoffs;
        for (int q = 0; q < p.n_near; q++) {
            const int e = p.entries[p.list_first[par] + q];
            listed.insert({entry_dx(e), entry_dy(e), entry_dz(e)});
            hoffs.insert(p.hoff_near[p.list_first[par] + q]);
        }
        if (listed != stencil) bad++;
        for (int n = 0; n < 16; n++) {
            const int c = near2_code(n);
            const int dx = c % 5 - 2, dy = (c / 5) % 5 - 2, dz = c / 25 - 2;
            if (!hoffs.count(halo_index(px + dx, py + dy, pz + dz, 2))) bad++;
            if (!hoffs.count(halo_index(px - dx, py - dy, pz - dz, 2))) bad++;
        }
    }
    std::printf("%d\n", bad);
    return bad != 0;
}
