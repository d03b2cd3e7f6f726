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

template <class T> __device__ __forceinline__ const T* mom_of(const DevTree& t);
template <> __device__ __forceinline__ const double* mom_of<double>(const DevTree& t) { return t.mom64; }
template <> __device__ __forceinline__ const float* mom_of<float>(const DevTree& t) { return t.mom32; }

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
    const T* __restrict__ mom = mom_of<T>(t);
    const T dax = mom[N + cell], day = mom[2 * N + cell], daz = mom[3 * N + cell];
    T inv_ma = T(0.0), a3[10], ta[3];
    if (FULL && AM) {
        inv_ma = T(1.0 / t.mom64[cell]);
#pragma unroll
        for (int r = 0; r < 10; r++) a3[r] = mom[(10 + r) * N + cell];
        ta[0] = a3[0] + a3[3] + a3[5];
        ta[1] = a3[1] + a3[6] + a3[8];
        ta[2] = a3[2] + a3[7] + a3[9];
    }
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
                const T m = mom[sc];
                A.L0 = fma_(m, a, A.L0);
                A.L1[0] = fma_(m, b, A.L1[0]);
                A.L1[1] = fma_(m, c, A.L1[1]);
                A.L1[2] = fma_(m, d, A.L1[2]);
            }
            continue;
        }
        if (FULL && !sleaf && entry_near(e)) continue;  // resolved at the next level
        // R' = X_A - X_B in cell units: the source sits at offset d from the target
        const T x = (dax - mom[N + sc]) - T(dx);
        const T y = (day - mom[2 * N + sc]) - T(dy);
        const T z = (daz - mom[3 * N + sc]) - T(dz);
        const T m = mom[sc];
        if (sleaf) {
            m2l_pair<T, FULL, false, AM>(x, y, z, m, nullptr, nullptr, m * inv_ma, a3, ta, A);
        } else {
            T b2[6], b3[10];
#pragma unroll
            for (int r = 0; r < 6; r++) b2[r] = mom[(4 + r) * N + sc];
#pragma unroll
            for (int r = 0; r < 10; r++) b3[r] = mom[(10 + r) * N + sc];
            m2l_pair<T, FULL, true, AM>(x, y, z, m, b2, b3, m * inv_ma, a3, ta, A);
        }
    }
    // scale to physical units: L^(n) * (-G h^-(n+1)), correction * -(G/6) h^-2
    const double hi = (double)(8 << L) / t.size;
    const double s1 = -G * hi, s2 = s1 * hi, s3 = s2 * hi, s4 = s3 * hi;
    double* loc = t.loc;
    atomicAdd(loc + cell, s1 * ((double)A.L0 + n0));
    atomicAdd(loc + N + cell, s2 * ((double)A.L1[0] + n1));
    atomicAdd(loc + 2 * N + cell, s2 * ((double)A.L1[1] + n2));
    atomicAdd(loc + 3 * N + cell, s2 * ((double)A.L1[2] + n3));
    if (FULL) {
        const double d1 = (double)A.d1;
        atomicAdd(loc + 4 * N + cell, s3 * ((double)A.L2[0] + d1));
        atomicAdd(loc + 5 * N + cell, s3 * (double)A.L2[1]);
        atomicAdd(loc + 6 * N + cell, s3 * (double)A.L2[2]);
        atomicAdd(loc + 7 * N + cell, s3 * ((double)A.L2[3] + d1));
        atomicAdd(loc + 8 * N + cell, s3 * (double)A.L2[4]);
        atomicAdd(loc + 9 * N + cell, s3 * ((double)A.L2[5] + d1));
        const double Vx = (double)A.V[0], Vy = (double)A.V[1], Vz = (double)A.V[2];
        // Kronecker part of L3: delta_ij V_k + delta_ik V_j + delta_jk V_i
        const double k3[10] = {3 * Vx, Vy, Vz, Vx, 0.0, Vx, 3 * Vy, Vz, Vy, 3 * Vz};
#pragma unroll
        for (int r = 0; r < 10; r++) atomicAdd(loc + (10 + r) * N + cell, s4 * ((double)A.L3[r] + k3[r]));
    }
    if (AM) {
        const double sa = -(G / 6.0) * hi * hi;
#pragma unroll
        for (int a = 0; a < 3; a++) atomicAdd(loc + (20 + a) * N + cell, sa * (double)A.S[a]);
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
