// Cell-to-cell interactions of every level of the octree in one persistent
// launch (the stencil approach of Sec. 5.5; the multipole interactions with
// the angular-momentum correction of Sec. 4.3.1).
//
// Work decomposition: a work item is 32 target cells of one node (one parity
// class, one half in z) and a contiguous range of that parity's stencil
// list (near offsets first, then the far offsets whose parents are near).
// One warp owns one item at a time and fetches the next from a global
// counter (longest items first), so levels with very different node counts
// and costs share one launch without level barriers: the interactions of
// level L need only the moments, which the upward pass has finished.
//
// Per (target A, source B) pair, decided per lane:
//   both leaf cells           -> done by the lattice kernel (lattice.cu) for
//                                leaf nodes of level >= 1; for a leaf root
//                                here, from the same table (R = -d h exactly,
//                                1/|d| and D1(-d) = d/|d|^3, 4 FMAs)
//   near, both interior       -> skipped (resolved one level down)
//   otherwise                 -> M2L of order 3 + correction (pair_formula.cuh)
// Each lane accumulates in registers (FP64, or FP32 for the bulk form with
// the near leaf pairs kept in FP64) and adds its sums once per item into the
// cell's FP64 expansion with atomics, scaled to physical units.
#include <type_traits>

#include "kernels.hpp"
#include "items.cuh"
#include "pair_formula.cuh"

namespace otfmm {

namespace {


__device__ __forceinline__ void tab_of(const DevPlan& p, int k, double& a, double& b, double& c,
                                       double& d) {
    const double2 v0 = __ldg(p.tab64 + 2 * k), v1 = __ldg(p.tab64 + 2 * k + 1);
    a = v0.x; b = v0.y; c = v1.x; d = v1.y;
}
__device__ __forceinline__ void tab_of(const DevPlan& p, int k, float& a, float& b, float& c,
                                       float& d) {
    const float4 v = __ldg(p.tab32 + k);
    a = v.x; b = v.y; c = v.z; d = v.w;
}

constexpr int kMaxWarps = 16;

// Source/target loads from the per-cell records (head = m, dX; tail = M2,
// M3, the M3 trace vector and trace(M2)): FP64 records of 24 doubles hold the
// traces, FP32 records of 20 floats do not.
__device__ __forceinline__ void load_head(const DevTree& t, long long c, double& m, double& x,
                                          double& y, double& z) {
    const double2* p = reinterpret_cast<const double2*>(t.rec64 + c * kRec);
    const double2 a = __ldg(p), b = __ldg(p + 1);
    m = a.x;
    x = a.y;
    y = b.x;
    z = b.y;
}
__device__ __forceinline__ void load_head(const DevTree& t, long long c, float& m, float& x,
                                          float& y, float& z) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(t.mom32 + c * kMom));
    m = v.x;
    x = v.y;
    y = v.z;
    z = v.w;
}
__device__ __forceinline__ void load_tail(const DevTree& t, long long c, double* b2, double* b3,
                                          double* bt) {
    const double2* p = reinterpret_cast<const double2*>(t.rec64 + c * kRec);
    double v[20];
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const double2 q = __ldg(p + 2 + r);
        v[2 * r] = q.x;
        v[2 * r + 1] = q.y;
    }
#pragma unroll
    for (int r = 0; r < 6; r++) b2[r] = v[r];
#pragma unroll
    for (int r = 0; r < 10; r++) b3[r] = v[6 + r];
#pragma unroll
    for (int r = 0; r < 4; r++) bt[r] = v[16 + r];
}
__device__ __forceinline__ void load_tail(const DevTree& t, long long c, float* b2, float* b3,
                                          float* bt) {
    // 80-byte FP32 records: the traces are cheaper to form here than to load
    const float4* p = reinterpret_cast<const float4*>(t.mom32 + c * kMom);
    const float4 v1 = __ldg(p + 1), v2 = __ldg(p + 2), v3 = __ldg(p + 3), v4 = __ldg(p + 4);
    b2[0] = v1.x; b2[1] = v1.y; b2[2] = v1.z; b2[3] = v1.w; b2[4] = v2.x; b2[5] = v2.y;
    b3[0] = v2.z; b3[1] = v2.w; b3[2] = v3.x; b3[3] = v3.y; b3[4] = v3.z; b3[5] = v3.w;
    b3[6] = v4.x; b3[7] = v4.y; b3[8] = v4.z; b3[9] = v4.w;
    bt[0] = b3[0] + b3[3] + b3[5];
    bt[1] = b3[1] + b3[6] + b3[8];
    bt[2] = b3[2] + b3[7] + b3[9];
    bt[3] = b2[0] + b2[3] + b2[5];
}
// The target's octupole per unit mass, M3_A / m_A, and its trace vector
// (the correction's mass ratio, applied once per target in FP64); zero for a
// target of zero mass (whose M3 is zero for non-negative densities).  The
// FP64 form divides here; the FP32 form reads the FP32 records that the
// upward pass formed in FP64.
__device__ __forceinline__ void load_octupole_per_mass(const DevTree& t, long long c, double* a3,
                                                       double* ta) {
    const double2* p = reinterpret_cast<const double2*>(t.rec64 + c * kRec);
    const double m = __ldg(t.rec64 + c * kRec);
    const double r = m != 0.0 ? 1.0 / m : 0.0;
    double v[14];
#pragma unroll
    for (int q = 0; q < 7; q++) {
        const double2 w = __ldg(p + 5 + q);
        v[2 * q] = w.x;
        v[2 * q + 1] = w.y;
    }
#pragma unroll
    for (int q = 0; q < 10; q++) a3[q] = r * v[q];
#pragma unroll
    for (int q = 0; q < 3; q++) ta[q] = r * v[10 + q];
}
__device__ __forceinline__ void load_octupole_per_mass(const DevTree& t, long long c, float* a3,
                                                       float* ta) {
    const float4* p = reinterpret_cast<const float4*>(t.oct32 + c * kOct);
    const float4 v0 = __ldg(p), v1 = __ldg(p + 1), v2 = __ldg(p + 2), v3 = __ldg(p + 3);
    a3[0] = v0.x; a3[1] = v0.y; a3[2] = v0.z; a3[3] = v0.w; a3[4] = v1.x;
    a3[5] = v1.y; a3[6] = v1.z; a3[7] = v1.w; a3[8] = v2.x; a3[9] = v2.y;
    ta[0] = v2.z; ta[1] = v2.w; ta[2] = v3.x;
}
__device__ __forceinline__ void load_off(const DevPlan& p, int k, double& x, double& y, double& z) {
    const double2 a = __ldg(p.off64 + 2 * k), b = __ldg(p.off64 + 2 * k + 1);
    x = a.x;
    y = a.y;
    z = b.x;
}
__device__ __forceinline__ void load_off(const DevPlan& p, int k, float& x, float& y, float& z) {
    const float4 a = __ldg(p.off32 + k);
    x = a.x;
    y = a.y;
    z = a.z;
}

// Scales a partial sum to physical units and widens it: the FP64 form
// multiplies in FP64; the FP32 form multiplies by the scale rounded to FP32
// (one more rounding of the size of the sum's own) and widens exactly.
__device__ __forceinline__ double scaled(double v, double s) { return s * v; }
__device__ __forceinline__ double scaled(float v, float s) { return widen(v * s); }
__device__ __forceinline__ const double* scales_of(const LevelScales& sc, int L, double) { return sc.s64[L]; }
__device__ __forceinline__ const float* scales_of(const LevelScales& sc, int L, float) { return sc.s32[L]; }

// Small non-negative integer (< 2^22) to T without a conversion
// instruction: for FP32, 2^23 + n is the float whose fraction bits are n.
__device__ __forceinline__ double small_int(int n, double) { return (double)n; }
__device__ __forceinline__ float small_int(int n, float) {
    return __int_as_float(0x4b000000 | n) - 8388608.0f;
}

// FP32 partial sums of the wide form span at most kFlush32 pairs of a lane:
// their rounding error grows with the summation length.
constexpr int kFlush32 = 64;

template <class T, bool FULL, bool AM>
__device__ __forceinline__ void run_item(const DevTree& t, const DevPlan& p, const int4 it,
                                         const int lane, const int* s_nb, const int* s_lf,
                                         const LevelScales& sc) {
    const int node = it.x;
    const int L = item_level(it);
    int i, j, k;
    item_cell(p, it, lane, i, j, k);
    const long long N = t.n_cells;
    const long long cell = (long long)node * kCells + i + 8 * j + 64 * k;
    T ma, dax, day, daz;
    load_head(t, cell, ma, dax, day, daz);
    Acc<T> A;
    acc_zero(A);
    double n0 = 0.0, n1 = 0.0, n2 = 0.0, n3 = 0.0;  // FP64 near leaf pairs (bulk form)
    // Adds the partial sums into the cell's FP64 expansion with atomics,
    // scaled to physical units: L^(n) * (-G h^-(n+1)), correction * -(G/6) h^-2,
    // with the level's factors in the accumulators' type.
    auto flush = [&]() {
        const T* sl = scales_of(sc, L, T(0));
        // (the L2, L3 and correction sums are held without their radial
        // constants kAccL2, kAccL3, kAccCor)
        const T s1 = sl[0], s2 = sl[1], s3 = sl[2] * T(kAccL2), s4 = sl[3] * T(kAccL3);
        double* loc = t.loc;
        if (sizeof(T) == 4 && L == 0 && !FULL) {
            // a leaf root: its near pairs were summed in FP64
            const double s1d = sc.s64[0][0], s2d = sc.s64[0][1];
            atomicAdd(loc + cell, scaled(A.L0, s1) + s1d * n0);
            atomicAdd(loc + N + cell, scaled(A.L1[0], s2) + s2d * n1);
            atomicAdd(loc + 2 * N + cell, scaled(A.L1[1], s2) + s2d * n2);
            atomicAdd(loc + 3 * N + cell, scaled(A.L1[2], s2) + s2d * n3);
        } else {
            atomicAdd(loc + cell, scaled(A.L0, s1));
            atomicAdd(loc + N + cell, scaled(A.L1[0], s2));
            atomicAdd(loc + 2 * N + cell, scaled(A.L1[1], s2));
            atomicAdd(loc + 3 * N + cell, scaled(A.L1[2], s2));
        }
        if (FULL) {
            finish_acc(A);  // Kronecker parts of L2 and L3 from their traces
#pragma unroll
            for (int r = 0; r < 6; r++) atomicAdd(loc + (4 + r) * N + cell, scaled(A.L2[r], s3));
#pragma unroll
            for (int r = 0; r < 10; r++) atomicAdd(loc + (10 + r) * N + cell, scaled(A.L3[r], s4));
        }
        if (AM) {
            // a_c = -(G/6) h^-2 (S - P), P from A4 and the target's octupole
            // per unit mass (loaded here, not held across the pair loop)
            const T sa = sl[4] * T(kAccCor);
            T P[3] = {T(0.0), T(0.0), T(0.0)};
            if (FULL) {
                T a3[10], ta[3];
                load_octupole_per_mass(t, cell, a3, ta);
                correction_target(A, a3, ta, P);
                if constexpr (std::is_same<T, double>::value) {
                    // the adjoint's forward pass keeps the quartic sum
                    if (p.a4_out)
#pragma unroll
                        for (int r = 0; r < 15; r++)
                            atomicAdd(p.a4_out + r * N + cell, A.A4[r] * kAccCor);
                }
            }
#pragma unroll
            for (int a = 0; a < 3; a++) atomicAdd(loc + (20 + a) * N + cell, scaled(A.S[a] - P[a], sa));
        }
    };
    // One pair with a source of kind 2 (a leaf cell) or 3 (an interior cell)
    // in cell src, stencil entry ent.  With multi (some lane of the warp has
    // an interior source) a leaf source takes the multipole formula with
    // zero moments: the same sums, in the warp's single pass.
    auto pair_at = [&](int kind, bool multi, long long src, int ent) {
        T m, bx, by, bz, ox, oy, oz;
        load_head(t, src, m, bx, by, bz);
        load_off(p, ent, ox, oy, oz);
        // R' = X_A - X_B in cell units: the source sits at offset d from the target
        const T x = (dax - bx) - ox;
        const T y = (day - by) - oy;
        const T z = (daz - bz) - oz;
        if (!multi) {
            m2l_pair<T, FULL, false, AM>(x, y, z, m, nullptr, nullptr, nullptr, A);
            return;
        }
        T b2[6], b3[10], bt[4];
        if (kind == 3) {
            load_tail(t, src, b2, b3, bt);
        } else {
#pragma unroll
            for (int r = 0; r < 6; r++) b2[r] = T(0.0);
#pragma unroll
            for (int r = 0; r < 10; r++) b3[r] = T(0.0);
#pragma unroll
            for (int r = 0; r < 4; r++) bt[r] = T(0.0);
        }
        m2l_pair<T, FULL, true, AM>(x, y, z, m, b2, b3, bt, A);
    };
    if (FULL && item_list(it) == kRootList) {
        // the interior root: sources are the root's own cells [z, w), the
        // same cell for every lane (a broadcast load); a pair is far iff
        // |d|^2 > near_d2, and near pairs of two interior cells descend
        const int root = it.x;
        const T fi = small_int(i, T(0)), fj = small_int(j, T(0)), fk = small_int(k, T(0));
#pragma unroll 1
        for (int s = it.z; s < it.w; s++) {
            const int sx = s & 7, sy = (s >> 3) & 7, sz = s >> 6;
            const int dx = sx - i, dy = sy - j, dz = sz - k;
            T m, bx, by, bz, b2[6], b3[10], bt[4];
            const long long sc = (long long)root * kCells + s;
            load_head(t, sc, m, bx, by, bz);
            load_tail(t, sc, b2, b3, bt);
            if (dx * dx + dy * dy + dz * dz <= p.near_d2) continue;
            // R' = (t + dX_A) - (s + dX_B) in cell units
            const T x = (fi + dax) - (small_int(sx, T(0)) + bx);
            const T y = (fj + day) - (small_int(sy, T(0)) + by);
            const T z = (fk + daz) - (small_int(sz, T(0)) + bz);
            m2l_pair<T, FULL, true, AM>(x, y, z, m, b2, b3, bt, A);
        }
    } else if (item_list(it) == kGroupList) {
        // grouped item: every lane walks its own list and computes its pairs
        // one after another; the warp runs while any lane has a pair left.
        // The wide FP32 form adds a lane's FP32 partial sums to the FP64
        // expansion every kFlush32 pairs.
        const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
        const int base = __ldg(p.list_first + par);
        const int qend = min(it.z >> 16, __ldg(p.list_len + par));
        int q = it.z & 0xffff;
        int since = 0;
#pragma unroll 1
        for (;;) {
            int nb = 0, lc = 0;
            const int kind = next_grouped<FULL>(p, s_nb, s_lf, base, qend, i, j, k, q, nb, lc);
            if (!__any_sync(0xffffffffu, kind != 0)) break;
            const bool multi = __any_sync(0xffffffffu, kind == 3);
            if (kind != 0) {
                pair_at(kind, multi, (long long)nb * kCells + lc, base + q);
                if (sizeof(T) == 4 && ++since == kFlush32) {
                    flush();
                    acc_zero(A);
                    since = 0;
                }
            }
            q++;
        }
    } else {
    const int base = p.list_first[item_list(it)];
#pragma unroll 1
    for (int pos = it.z; pos < it.w; pos++) {
        const int q = __ldg(p.item_entries + pos);
        const int e = __ldg(p.entries + base + q);
        const int dx = entry_dx(e), dy = entry_dy(e), dz = entry_dz(e);
        const int sx = i + dx, sy = j + dy, sz = k + dz;
        const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
        const int nb = s_nb[slot];
        const bool sleaf = s_lf[slot] != 0;
        // 0: no pair (outside the domain, covered by a coarser leaf, a
        // leaf-leaf pair of level >= 1 for the lattice kernel, or a near
        // pair of two interior cells resolved at the next level); 1: two
        // point masses of a leaf root; 2: a leaf source; 3: an interior one
        int kind = 0;
        if (nb >= 0) {
            if (!FULL && sleaf) kind = L > 0 ? 0 : 1;
            else if (!(FULL && !sleaf && entry_near(e))) kind = sleaf ? 2 : 3;
        }
        // where the warp holds both leaf and interior sources, the leaf ones
        // take the multipole formula with zero moments (the same sums) rather
        // than a second, divergent pass
        const bool multi = __any_sync(0xffffffffu, kind == 3);
        if (kind == 0) continue;
        const long long sc = (long long)nb * kCells + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
        if (kind == 1) {
            // two point masses on the lattice (a leaf root)
            if (sizeof(T) == 4 && entry_near(e)) {
                double a, b, c, d;
                tab_of(p, base + q, a, b, c, d);
                const double m = t.mom64[sc];
                n0 = fma(m, a, n0);
                n1 = fma(m, b, n1);
                n2 = fma(m, c, n2);
                n3 = fma(m, d, n3);
            } else {
                T a, b, c, d;
                tab_of(p, base + q, a, b, c, d);
                T m, u0, u1, u2;
                load_head(t, sc, m, u0, u1, u2);
                A.L0 = fma_(m, a, A.L0);
                A.L1[0] = fma_(m, b, A.L1[0]);
                A.L1[1] = fma_(m, c, A.L1[1]);
                A.L1[2] = fma_(m, d, A.L1[2]);
            }
            continue;
        }
        pair_at(kind, multi, sc, base + q);
    }
    }
    flush();
}

// FP32-bulk form: one item with the pair split by precision (m2l_pair_split):
// the monopole part of every pair and the correction's sums in FP64, the
// source's quadrupole and octupole contractions in FP32 (partial sums of at
// most kFlush32 pairs, then added to the FP64 sums).  Leaf-leaf pairs of a
// leaf root are monopole pairs: FP64 from the lattice table.
template <bool FULL, bool AM>
__device__ __forceinline__ void run_item_split(const DevTree& t, const DevPlan& p, const int4 it,
                                               const int lane, const int* s_nb, const int* s_lf,
                                               const LevelScales& sc) {
    const int node = it.x;
    const int L = item_level(it);
    int i, j, k;
    item_cell(p, it, lane, i, j, k);
    const long long N = t.n_cells;
    const long long cell = (long long)node * kCells + i + 8 * j + 64 * k;
    double ma, dax, day, daz;
    load_head(t, cell, ma, dax, day, daz);
    float maf, daxf, dayf, dazf;
    load_head(t, cell, maf, daxf, dayf, dazf);
    SplitAcc<double, float> A;
    split_zero(A);
    int since = 0;  // pairs summed in the FP32 partial sums
    auto pair = [&](double x, double y, double z, double m, float xf, float yf, float zf,
                    long long src, bool sleaf) {
        if (sleaf) {
            m2l_pair_split<double, float, FULL, false, AM>(x, y, z, m, 0.f, 0.f, 0.f, nullptr, nullptr,
                                                           nullptr, A);
        } else {
            float b2[6], b3[10], bt[4];
            load_tail(t, src, b2, b3, bt);
            m2l_pair_split<double, float, FULL, true, AM>(x, y, z, m, xf, yf, zf, b2, b3, bt, A);
            if (++since == kFlush32) {
                flush_split(A);
                since = 0;
            }
        }
    };
    // A pair through a stencil entry (kinds and multi as in run_item): R in
    // FP64 from the FP64 records, and in FP32 from the FP32 ones for the
    // multipole part.
    auto pair_at = [&](int kind, bool multi, long long src, int ent) {
        double m, bx, by, bz, ox, oy, oz;
        load_head(t, src, m, bx, by, bz);
        load_off(p, ent, ox, oy, oz);
        const double x = (dax - bx) - ox, y = (day - by) - oy, z = (daz - bz) - oz;
        if (!multi) {
            m2l_pair_split<double, float, FULL, false, AM>(x, y, z, m, 0.f, 0.f, 0.f, nullptr, nullptr,
                                                           nullptr, A);
            return;
        }
        float mf, bxf, byf, bzf, oxf, oyf, ozf;
        load_head(t, src, mf, bxf, byf, bzf);
        load_off(p, ent, oxf, oyf, ozf);
        const float xf = (daxf - bxf) - oxf, yf = (dayf - byf) - oyf, zf = (dazf - bzf) - ozf;
        float b2[6], b3[10], bt[4];
        if (kind == 3) {
            load_tail(t, src, b2, b3, bt);
        } else {
#pragma unroll
            for (int r = 0; r < 6; r++) b2[r] = 0.f;
#pragma unroll
            for (int r = 0; r < 10; r++) b3[r] = 0.f;
#pragma unroll
            for (int r = 0; r < 4; r++) bt[r] = 0.f;
        }
        m2l_pair_split<double, float, FULL, true, AM>(x, y, z, m, xf, yf, zf, b2, b3, bt, A);
        if (++since == kFlush32) {
            flush_split(A);
            since = 0;
        }
    };
    if (FULL && item_list(it) == kRootList) {
        // the interior root: sources are the root's own cells [z, w)
        const int root = it.x;
#pragma unroll 1
        for (int s = it.z; s < it.w; s++) {
            const int sx = s & 7, sy = (s >> 3) & 7, sz = s >> 6;
            const int dx = sx - i, dy = sy - j, dz = sz - k;
            if (dx * dx + dy * dy + dz * dz <= p.near_d2) continue;
            const long long src = (long long)root * kCells + s;
            double m, bx, by, bz;
            load_head(t, src, m, bx, by, bz);
            float mf, bxf, byf, bzf;
            load_head(t, src, mf, bxf, byf, bzf);
            // R' = (t + dX_A) - (s + dX_B) in cell units
            const double x = (dax - bx) - (double)dx, y = (day - by) - (double)dy, z = (daz - bz) - (double)dz;
            const float xf = (daxf - bxf) - (float)dx, yf = (dayf - byf) - (float)dy,
                        zf = (dazf - bzf) - (float)dz;
            pair(x, y, z, m, xf, yf, zf, src, false);
        }
    } else if (item_list(it) == kGroupList) {
        // grouped item: every lane walks its own list (see run_item)
        const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
        const int base = __ldg(p.list_first + par);
        const int qend = min(it.z >> 16, __ldg(p.list_len + par));
        int q = it.z & 0xffff;
#pragma unroll 1
        for (;;) {
            int nb = 0, lc = 0;
            const int kind = next_grouped<FULL>(p, s_nb, s_lf, base, qend, i, j, k, q, nb, lc);
            if (!__any_sync(0xffffffffu, kind != 0)) break;
            const bool multi = __any_sync(0xffffffffu, kind == 3);
            if (kind != 0) pair_at(kind, multi, (long long)nb * kCells + lc, base + q);
            q++;
        }
    } else {
        const int base = p.list_first[item_list(it)];
#pragma unroll 1
        for (int pos = it.z; pos < it.w; pos++) {
            const int q = __ldg(p.item_entries + pos);
            const int e = __ldg(p.entries + base + q);
            const int dx = entry_dx(e), dy = entry_dy(e), dz = entry_dz(e);
            const int sx = i + dx, sy = j + dy, sz = k + dz;
            const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
            const int nb = s_nb[slot];
            const bool sleaf = s_lf[slot] != 0;
            // pair kinds as in run_item: 0 none, 1 point masses of a leaf
            // root, 2 leaf source, 3 interior source
            int kind = 0;
            if (nb >= 0) {
                if (!FULL && sleaf) kind = L > 0 ? 0 : 1;
                else if (!(FULL && !sleaf && entry_near(e))) kind = sleaf ? 2 : 3;
            }
            // leaf sources of a warp that also holds interior ones take the
            // multipole formula with zero moments, in the same pass
            const bool multi = __any_sync(0xffffffffu, kind == 3);
            if (kind == 0) continue;
            const long long src = (long long)nb * kCells + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
            if (kind == 1) {
                // two point masses on the lattice (a leaf root), FP64
                double a, b, c, d;
                tab_of(p, base + q, a, b, c, d);
                const double m = t.mom64[src];
                A.L0 = fma(m, a, A.L0);
                A.L1[0] = fma(m, b, A.L1[0]);
                A.L1[1] = fma(m, c, A.L1[1]);
                A.L1[2] = fma(m, d, A.L1[2]);
                continue;
            }
            pair_at(kind, multi, src, base + q);
        }
    }
    flush_split(A);
    // to physical units, one atomic per component
    const double* sl = sc.s64[L];
    double* loc = t.loc;
    atomicAdd(loc + cell, sl[0] * A.L0);
    atomicAdd(loc + N + cell, sl[1] * A.L1[0]);
    atomicAdd(loc + 2 * N + cell, sl[1] * A.L1[1]);
    atomicAdd(loc + 3 * N + cell, sl[1] * A.L1[2]);
    if (FULL) {
        finish_split(A);
#pragma unroll
        for (int r = 0; r < 6; r++) atomicAdd(loc + (4 + r) * N + cell, sl[2] * A.L2[r]);
#pragma unroll
        for (int r = 0; r < 10; r++) atomicAdd(loc + (10 + r) * N + cell, sl[3] * A.L3[r]);
    }
    if (AM) {
        double P[3] = {0.0, 0.0, 0.0};
        if (FULL) {
            double a3[10], ta[3];
            load_octupole_per_mass(t, cell, a3, ta);
            correction_target_split(A, a3, ta, P);
        }
#pragma unroll
        for (int a = 0; a < 3; a++) atomicAdd(loc + (20 + a) * N + cell, sl[4] * (A.S[a] - P[a]));
    }
}

// Persistent launch of the FP32-bulk form (the split pair).
__global__ void __launch_bounds__(128, 3) k_interact_split(DevTree t, DevPlan p, LevelScales sc, int am) {
    __shared__ int s_nb[kMaxWarps][28];
    __shared__ int s_lf[kMaxWarps][28];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(p.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= p.n_items) break;
        const int4 it = __ldg(p.items + item);
        if (lane < 27) {
            const int nb = t.nbr[(long long)it.x * 27 + lane];
            s_nb[w][lane] = nb;
            s_lf[w][lane] = nb >= 0 ? (t.node_leaf[nb] >= 0) : 0;
        }
        __syncwarp();
        const bool full = t.node_leaf[it.x] < 0;
        if (full) {
            if (am) run_item_split<true, true>(t, p, it, lane, s_nb[w], s_lf[w], sc);
            else run_item_split<true, false>(t, p, it, lane, s_nb[w], s_lf[w], sc);
        } else {
            if (am) run_item_split<false, true>(t, p, it, lane, s_nb[w], s_lf[w], sc);
            else run_item_split<false, false>(t, p, it, lane, s_nb[w], s_lf[w], sc);
        }
        __syncwarp();
    }
}

template <class T>
__global__ void __launch_bounds__(128, std::is_same<T, double>::value ? 3 : 1)
    k_interact(DevTree t, DevPlan p, LevelScales sc, int am) {
    __shared__ int s_nb[kMaxWarps][28];
    __shared__ int s_lf[kMaxWarps][28];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(p.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= p.n_items) break;
        const int4 it = __ldg(p.items + item);
        if (lane < 27) {
            const int nb = t.nbr[(long long)it.x * 27 + lane];
            s_nb[w][lane] = nb;
            s_lf[w][lane] = nb >= 0 ? (t.node_leaf[nb] >= 0) : 0;
        }
        __syncwarp();
        const bool full = t.node_leaf[it.x] < 0;
        if (!full && p.interior_only) continue;
        if (full) {
            if (am) run_item<T, true, true>(t, p, it, lane, s_nb[w], s_lf[w], sc);
            else run_item<T, true, false>(t, p, it, lane, s_nb[w], s_lf[w], sc);
        } else {
            if (am) run_item<T, false, true>(t, p, it, lane, s_nb[w], s_lf[w], sc);
            else run_item<T, false, false>(t, p, it, lane, s_nb[w], s_lf[w], sc);
        }
        __syncwarp();
    }
}

}  // namespace

int configure_interact() {
    // Half of the unified L1/shared memory as shared memory: the general
    // kernels read their source records through L1, and measured on the
    // level-3 and level-6 binaries beside the lattice kernels (which ask for
    // the largest carveout) a 50 % split was fastest in both forms (no
    // preference, 0 % and 100 % were up to 15 % slower).
    const int carve = 50;
    if (cudaFuncSetAttribute(k_interact<float>, cudaFuncAttributePreferredSharedMemoryCarveout, carve) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_interact<double>, cudaFuncAttributePreferredSharedMemoryCarveout, carve) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_interact_split, cudaFuncAttributePreferredSharedMemoryCarveout, carve) !=
            cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}

void launch_interact(const DevTree& t, const DevPlan& p, int precision, double G, int am,
                     int ctas, int warps_per_cta, cudaStream_t s) {
    if (warps_per_cta > 4) warps_per_cta = 4;
    const LevelScales sc = level_scales(t.inv_side8, G);
    // every form takes the grouped items where the plan has them
    DevPlan g = p;
    if (p.items_grp) {
        g.items = p.items_grp;
        g.n_items = p.n_items_grp;
    }
    if (precision == kPrecWide)
        k_interact<float><<<ctas, 32 * warps_per_cta, 0, s>>>(t, g, sc, am);
    else if (precision == kPrecBulk)
        k_interact_split<<<ctas, 32 * warps_per_cta, 0, s>>>(t, g, sc, am);
    else
        k_interact<double><<<ctas, 32 * warps_per_cta, 0, s>>>(t, g, sc, am);
}

}  // namespace otfmm
