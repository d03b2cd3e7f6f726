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
#include "kernels.hpp"
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
// The target's octupole per unit mass, M3_A / m_A, and its trace vector,
// formed in FP64 once per target (the correction's mass ratio); zero for a
// target of zero mass (whose M3 is zero for non-negative densities).
template <class T>
__device__ __forceinline__ void load_octupole_per_mass(const DevTree& t, long long c, T* a3, T* ta) {
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
    for (int q = 0; q < 10; q++) a3[q] = T(r * v[q]);
#pragma unroll
    for (int q = 0; q < 3; q++) ta[q] = T(r * v[10 + q]);
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
// (one more rounding of the size of the sum's own) and converts once.
__device__ __forceinline__ double scaled(double v, double s) { return s * v; }
__device__ __forceinline__ double scaled(float v, float s) { return (double)(v * s); }

template <class T, bool FULL, bool AM>
__device__ __forceinline__ void run_item(const DevTree& t, const DevPlan& p, const int4 it,
                                         const int lane, const int* s_nb, const int* s_lf,
                                         double G) {
    const int node = it.x;
    const int L = item_level(it), par = item_parity(it), half = item_half(it);
    const int i = 2 * (lane & 3) + (par & 1);
    const int j = 2 * ((lane >> 2) & 3) + ((par >> 1) & 1);
    const int k = 2 * (2 * half + (lane >> 4)) + (par >> 2);
    const long long N = t.n_cells;
    const long long cell = (long long)node * kCells + i + 8 * j + 64 * k;
    T ma, dax, day, daz;
    load_head(t, cell, ma, dax, day, daz);
    T a3[10], ta[4];
    if (FULL && AM) load_octupole_per_mass(t, cell, a3, ta);
    Acc<T> A;
    acc_zero(A);
    double n0 = 0.0, n1 = 0.0, n2 = 0.0, n3 = 0.0;  // FP64 near leaf pairs (bulk form)
    const int base = p.list_first[item_list(it)];
#pragma unroll 1
    for (int q = it.z; q < it.w; q++) {
        const int e = __ldg(p.entries + base + q);
        const int dx = entry_dx(e), dy = entry_dy(e), dz = entry_dz(e);
        const int sx = i + dx, sy = j + dy, sz = k + dz;
        const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
        const int nb = s_nb[slot];
        if (nb < 0) continue;  // outside the domain, or covered by a coarser leaf
        const bool sleaf = s_lf[slot] != 0;
        const long long sc = (long long)nb * kCells + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
        if (!FULL && sleaf) {
            if (L > 0) continue;  // leaf-leaf pairs of level >= 1: lattice kernel
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
        if (FULL && !sleaf && entry_near(e)) continue;  // resolved at the next level
        T m, bx, by, bz, ox, oy, oz;
        load_head(t, sc, m, bx, by, bz);
        load_off(p, base + q, ox, oy, oz);
        // R' = X_A - X_B in cell units: the source sits at offset d from the target
        const T x = (dax - bx) - ox;
        const T y = (day - by) - oy;
        const T z = (daz - bz) - oz;
        if (sleaf) {
            m2l_pair<T, FULL, false, AM>(x, y, z, m, nullptr, nullptr, nullptr, a3, ta, A);
        } else {
            T b2[6], b3[10], bt[4];
            load_tail(t, sc, b2, b3, bt);
            m2l_pair<T, FULL, true, AM>(x, y, z, m, b2, b3, bt, a3, ta, A);
        }
    }
    // scale to physical units: L^(n) * (-G h^-(n+1)), correction * -(G/6) h^-2
    const double hi = t.inv_side8 * (double)(1 << L);
    const double s1d = -G * hi, s2d = s1d * hi;
    // scale factors in the accumulators' type (converted once per item)
    const T s1 = T(s1d), s2 = T(s2d), s3 = T(s2d * hi), s4 = T(s2d * hi * hi);
    double* loc = t.loc;
    atomicAdd(loc + cell, scaled(A.L0, s1) + s1d * n0);
    atomicAdd(loc + N + cell, scaled(A.L1[0], s2) + s2d * n1);
    atomicAdd(loc + 2 * N + cell, scaled(A.L1[1], s2) + s2d * n2);
    atomicAdd(loc + 3 * N + cell, scaled(A.L1[2], s2) + s2d * n3);
    if (FULL) {
        finish_acc(A);  // Kronecker parts of L2 and L3 from their traces
#pragma unroll
        for (int r = 0; r < 6; r++) atomicAdd(loc + (4 + r) * N + cell, scaled(A.L2[r], s3));
#pragma unroll
        for (int r = 0; r < 10; r++) atomicAdd(loc + (10 + r) * N + cell, scaled(A.L3[r], s4));
    }
    if (AM) {
        // a_c = -(G/6) h^-2 (S - P)
        const T sa = T(-(G / 6.0) * hi * hi);
#pragma unroll
        for (int a = 0; a < 3; a++)
            atomicAdd(loc + (20 + a) * N + cell, scaled(FULL ? A.S[a] - A.P[a] : A.S[a], sa));
    }
}

template <class T>
__global__ void __launch_bounds__(128) k_interact(DevTree t, DevPlan p, double G, int am) {
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
            if (am) run_item<T, true, true>(t, p, it, lane, s_nb[w], s_lf[w], G);
            else run_item<T, true, false>(t, p, it, lane, s_nb[w], s_lf[w], G);
        } else {
            if (am) run_item<T, false, true>(t, p, it, lane, s_nb[w], s_lf[w], G);
            else run_item<T, false, false>(t, p, it, lane, s_nb[w], s_lf[w], G);
        }
        __syncwarp();
    }
}

}  // namespace

void launch_interact(const DevTree& t, const DevPlan& p, int precision, double G, int am,
                     int ctas, int warps_per_cta, cudaStream_t s) {
    if (warps_per_cta > 4) warps_per_cta = 4;
    if (precision == 1)
        k_interact<float><<<ctas, 32 * warps_per_cta, 0, s>>>(t, p, G, am);
    else
        k_interact<double><<<ctas, 32 * warps_per_cta, 0, s>>>(t, p, G, am);
}

}  // namespace otfmm
