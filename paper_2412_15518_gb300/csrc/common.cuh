// Shared device-side definitions of the GB300 FMM gravity library.
//
// Data layout in HBM (all levels concatenated, nodes in breadth-first order
// with the 8 children of a node contiguous in octant order x + 2y + 4z):
//   node arrays   [n_nodes]              level, leaf id (-1 interior), parent,
//                                        first child, 27 same-level neighbours
//   cell arrays   [component][n_cells]   structure of arrays, cell = node * 512
//                                        + i + 8 j + 64 k
//   moments       20 components: m, dX(3), M2(6), M3(10) in units of the cell's
//                 own side h (dX = centre of mass - cell centre, M2 / h^2,
//                 M3 / h^3); FP64 structure of arrays [20][n_cells]; FP64
//                 per-cell records [n_cells][24] (the 20 moments, the M3
//                 trace vector t_i = M3_ijj and trace(M2)) and FP32 records
//                 [n_cells][20], read by the interaction kernels (a source is
//                 a few 16-byte loads); FP32 leaf masses [n_cells] (the
//                 lattice kernel's halo); FP32 octupole per unit mass
//                 [n_cells][16] of interior cells (M3 / m, its trace vector;
//                 the correction's target term)
//   expansions    23 components: L0, L1(3), L2(6), L3(10), ac(3), physical
//                 units, FP64
// Packed symmetric index orders: M2/L2 = xx xy xz yy yz zz;
// M3/L3 = xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace otfmm {

constexpr int kCells = 512;      // 8^3 cells per node (Sec. 4.3.2)
constexpr int kMom = 20;         // moment components per cell
constexpr int kRec = 24;         // per-cell record: 20 moments, M3 trace vector, M2 trace
constexpr int kLoc = 23;         // expansion components per cell (+ correction)
constexpr int kOct = 16;         // per-cell FP32 octupole record: M3 / m (10), trace vector (3), pad
constexpr int kMaxLevels = 16;   // levels 0..15

// Precision forms (the OT_PRECISION_* codes of the C ABI): every step in
// FP64; the FP32-bulk form (monopole parts, correction and every sum in FP64,
// the source multipole contractions in FP32); the wide FP32 form (every
// per-pair multipole term in FP32, FP64 near pairs and sums).
constexpr int kPrecFP64 = 0;
constexpr int kPrecBulk = 1;
constexpr int kPrecWide = 2;

// Status word codes latched by kernels (never trapped).
constexpr int kStatusBadIndex = 1;
constexpr int kStatusBadDensity = 4;  // a hydro face state with density <= 0 or NaN
// (bit 2 is reserved: no kernel stages a bounded number of item entries)

// Device view of a tree and its current plan; passed by value to kernels.
struct DevTree {
    int n_levels;
    int n_nodes;
    int n_leaf;
    long long n_cells;          // n_nodes * 512
    double size;
    double origin[3];           // corner of the domain cube
    const int* node_level;      // [n_nodes]
    const int* node_leaf;       // [n_nodes] leaf id or -1
    const int* node_parent;     // [n_nodes] or -1
    const int* node_child;      // [n_nodes] first child or -1
    const int* node_xyz;        // [n_nodes][3] node coordinates at its level
    const int* nbr;             // [n_nodes][27] neighbour node or -1
    const int* level_first;     // [n_levels + 1] first node of each level
    double* mom64;              // [20][n_cells]
    double* rec64;              // [n_cells][24]
    float* mom32;               // [n_cells][20]
    float* m32;                 // [n_cells] leaf masses (FP32)
    float* oct32;               // [n_cells][16] interior cells: M3 / m, trace vector
    double inv_side8;           // 8 / size: 1/h at level 0
    double* loc;                // [23][n_cells]
    int* status;                // device status word
};

// Per-level factors from cell units to physical units, computed on the host
// for each solve (they hold G): s[L][n] = -G h_L^-(n+1) for the expansion
// orders n = 0..3, s[L][4] = -(G/6) h_L^-2 for the correction.
struct LevelScales {
    double s64[kMaxLevels][5];
    float s32[kMaxLevels][5];
};

inline LevelScales level_scales(double inv_side8, double G) {
    LevelScales r;
    for (int L = 0; L < kMaxLevels; L++) {
        const double hi = inv_side8 * (double)(1 << L);
        const double s1 = -G * hi, s2 = s1 * hi;
        const double v[5] = {s1, s2, s2 * hi, s2 * hi * hi, -(G / 6.0) * hi * hi};
        for (int n = 0; n < 5; n++) {
            r.s64[L][n] = v[n];
            r.s32[L][n] = (float)v[n];
        }
    }
    return r;
}

// Exact IEEE-754 binary32 -> binary64 widening by integer operations only
// (on this GPU the hardware conversion issues on the FP64 pipe, at 1/64 of
// the FP32 rate).  Normal numbers: the exponent is rebiased (127 -> 1023) and
// the 23-bit fraction moved to the top of the 52-bit one.  Subnormals
// (e = 0, f != 0): the fraction is shifted until its leading one reaches the
// implicit bit, and the exponent lowered by the shift.  Zeros keep their
// sign; infinities and NaNs get the all-ones exponent (a NaN keeps its
// payload with the quiet bit set).
__host__ __device__ __forceinline__ unsigned clz32(unsigned x) {
#ifdef __CUDA_ARCH__
    return (unsigned)__clz((int)x);
#else
    return x ? (unsigned)__builtin_clz(x) : 32u;
#endif
}
__host__ __device__ __forceinline__ double widen(float f) {
    unsigned u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    std::memcpy(&u, &f, sizeof u);
#endif
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xffu;
    unsigned m = u & 0x7fffffu;
    unsigned E = e + 896u;                          // normal: rebias
    if (e == 0u) {                                  // zero or subnormal
        const unsigned sh = clz32(m) - 8u;          // leading one to bit 23
        m = (m << sh) & 0x7fffffu;
        E = m == 0u && sh == 24u ? 0u : 897u - sh;  // a zero keeps E = 0
    }
    if (e == 0xffu) {                               // infinity or NaN
        E = 0x7ffu;
        if (m) m |= 0x400000u;                      // quiet NaN
    }
    const unsigned hi = sign | (E << 20) | (m >> 3);
    const unsigned lo = m << 29;
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)hi, (int)lo);
#else
    const unsigned long long b = ((unsigned long long)hi << 32) | lo;
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
#endif
}

#if defined(__CUDACC__)
// Asynchronous global -> shared copies (cp.async, through L1; 4, 8 or 16
// bytes, both addresses aligned to the size): the copy needs no register and
// nothing waits for it until cp.async.wait_group, so a thread can keep many
// in flight.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(a), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) { cp_async<16>(smem, gmem); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
#endif

// Stencil entries of a plan: int code = (dx+16) | (dy+16)<<5 | (dz+16)<<10 |
// near<<15; lists are contiguous ranges of the entry array.
struct DevPlan {
    const int* entries;         // [n_entries]
    const double2* tab64;       // [2 n_entries] (D0, D1x), (D1y, D1z) of the lattice offset
    const float4* tab32;        // [n_entries]
    const double2* off64;       // [2 n_entries] (dx, dy), (dz, 0) of each entry
    const float4* off32;        // [n_entries] (dx, dy, dz, 0)
    const int* list_first;      // [9] first entry of list 0..8 (8 = level 0)
    const int* list_len;        // [9]
    const int4* items;          // [n_items]
    const int* item_entries;    // forward items: list positions of their ranges
    int n_items;
    const int4* items_grp;      // [n_items_grp] the FP64 and FP32-bulk forms' items
    int n_items_grp;            //   (cells grouped by pair count, kGroupList)
    const unsigned short* grp_cells;  // 32 node-local cell indices per group
    int* counter;               // dynamic item counter of the persistent launch
    int near_d2;                // largest |d|^2 (cell units) of a near pair
    int interior_only;          // 1: skip the items of leaf targets (the adjoint's
                                // forward pass needs only interior expansions)
    double* a4_out;             // null, or [15][n_cells]: the FP64 general kernel
                                // adds each interior target's quartic sum
                                // sum_B m_B f4 R'^4 (cell units, packed as Acc::A4)
                                // here, which the adjoint's reverse pass reads
};

// List id of the items of an interior root: their range runs over the
// root's own 512 cells as sources instead of over stencil entries.
constexpr int kRootList = 9;
// List id of grouped items: 32 cells of one node of level >= 1 chosen by
// their number of pairs (grp_cells), each walking the list of its own parity
// class over the item's range of list positions.
constexpr int kGroupList = 10;

__host__ __device__ inline int pack_entry(int dx, int dy, int dz, int near) {
    return (dx + 16) | ((dy + 16) << 5) | ((dz + 16) << 10) | (near << 15);
}
__host__ __device__ inline int entry_dx(int e) { return (e & 31) - 16; }
__host__ __device__ inline int entry_dy(int e) { return ((e >> 5) & 31) - 16; }
__host__ __device__ inline int entry_dz(int e) { return ((e >> 10) & 31) - 16; }
__host__ __device__ inline int entry_near(int e) { return (e >> 15) & 1; }

// Shared-memory halo of leaf masses used by the lattice kernel: the cells of
// a node and of a margin w around it, split into 8 parity sub-halos so that a
// warp of same-parity targets reads consecutive words.  In a sub-halo the
// cell at node-local (x, y, z) (x in [-w, 8+w)) sits at
//   ((x+w)>>1) + kHaloPy ((y+w)>>1) + halo_pz(w) ((z+w)>>1),
// and sub-halo (x&1) + 2 (y&1) + 4 (z&1) starts at that index times
// halo_sub(w).  kHaloPy = 12 and halo_pz = 16 (mod 32) make the 32 lanes of a
// warp (4 x 4 x 2 targets) hit 32 distinct banks.
constexpr int kHaloPy = 12;
__host__ __device__ constexpr int halo_hh(int w) { return w + 4; }
__host__ __device__ constexpr int halo_pz(int w) {
    return kHaloPy * (w + 4) + (((16 - kHaloPy * (w + 4)) % 32) + 32) % 32;
}
__host__ __device__ constexpr int halo_sub(int w) { return halo_pz(w) * halo_hh(w); }
__host__ __device__ constexpr int halo_index(int x, int y, int z, int w) {
    return ((x & 1) + 2 * (y & 1) + 4 * (z & 1)) * halo_sub(w) + ((x + w) >> 1) +
           kHaloPy * ((y + w) >> 1) + halo_pz(w) * ((z + w) >> 1);
}

// Lattice part of a plan: halo offsets of every entry of the 8 parity lists
// (far halo of width w_far, near halo of width w_near), and the leaf nodes of
// level >= 1 whose leaf-leaf pairs the lattice kernel computes.
struct DevLattice {
    const int* hoff_far;        // [n_entries]
    const int* hoff_near;       // [n_entries] (near entries only)
    const int* nodes;           // [n_nodes_lattice]
    int n_nodes;
    int w_far, w_near;
    int n_near;
    int* counter;               // [2] node counters of the persistent CTAs (near/all, far)
    int n_far_max;              // largest far part of the 8 parity lists
    int far_table_smem;         // 1: the FP32 far kernel stages its tables in shared memory
};

// Work item: x = target node; y = level | parity << 8 | half << 11 | list << 12;
// z, w = range [k0, k1): of item_entries, whose values are positions in the
// list (forward launch); of the list itself (adjoint); of the root's cells
// (kRootList).  32 target cells per item: the
// cells of one parity class (px, py, pz) with z-index 2 (2 half + q) + pz,
// q in {0, 1}.  Grouped items (list kGroupList): y = level | group << 8 |
// list << 12, z = k0 | k1 << 16 (a range of list positions, each lane's
// clipped to its own list), w = index of the group's 32 cells in grp_cells.
__host__ __device__ inline int item_level(int4 it) { return it.y & 0xff; }
__host__ __device__ inline int item_parity(int4 it) { return (it.y >> 8) & 7; }
__host__ __device__ inline int item_half(int4 it) { return (it.y >> 11) & 1; }
__host__ __device__ inline int item_list(int4 it) { return (it.y >> 12) & 15; }

}  // namespace otfmm
