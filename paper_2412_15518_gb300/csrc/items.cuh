// Work-item helpers shared by the persistent interaction kernels (FP64,
// FP32-bulk and the tangent solve): the target cell of a lane, and the
// per-lane walk of a grouped item over the lane's own stencil list.
#pragma once

#include "common.cuh"

namespace otfmm {

// Node-local target cell (i, j, k) of a lane: from the item's parity class
// and half, or from its group's cell list (grouped items).
__device__ __forceinline__ void item_cell(const DevPlan& p, const int4 it, int lane, int& i, int& j,
                                          int& k) {
    if (item_list(it) == kGroupList) {
        const int c = __ldg(p.grp_cells + it.w + lane);
        i = c & 7;
        j = (c >> 3) & 7;
        k = c >> 6;
    } else {
        const int par = item_parity(it), half = item_half(it);
        i = 2 * (lane & 3) + (par & 1);
        j = 2 * ((lane >> 2) & 3) + ((par >> 1) & 1);
        k = 2 * (2 * half + (lane >> 4)) + (par >> 2);
    }
}

// Grouped items (level >= 1): moves q, this lane's position in the list of
// its own parity class, to its next pair in [q, qend) and returns the pair's
// kind (2: a leaf source, 3: an interior source; 0: no pair left), with the
// source's node and node-local cell.  An interior target pairs with every
// leaf source and with the far interior ones (near interior pairs descend to
// the next level); a leaf target only with interior sources (leaf-leaf
// pairs are the lattice kernel's).
template <bool FULL>
__device__ __forceinline__ int next_grouped(const DevPlan& p, const int* s_nb, const int* s_lf, int base,
                                            int qend, int i, int j, int k, int& q, int& nb, int& lc) {
    for (; q < qend; q++) {
        const int e = __ldg(p.entries + base + q);
        const int sx = i + entry_dx(e), sy = j + entry_dy(e), sz = k + entry_dz(e);
        const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
        const int n = s_nb[slot];
        if (n < 0) continue;  // outside the domain, or covered by a coarser leaf
        const bool sleaf = s_lf[slot] != 0;
        if (FULL ? (!sleaf && entry_near(e)) : sleaf) continue;
        nb = n;
        lc = (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
        return sleaf ? 2 : 3;
    }
    return 0;
}

}  // namespace otfmm
