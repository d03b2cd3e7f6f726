// Tangent (forward-mode derivative) of the solve: the time derivative of the
// potential and of the acceleration for a given rate of change of the
// densities (the FMM of Sec. 2 includes the time derivative of the
// potential, which the energy balance in the rotating frame needs, Sec.
// 4.3.1).  phi_dot = (d phi / d rho) . rho_dot, g_dot likewise: the exact
// derivative of the discrete solve, through the centres of mass and the
// correction's mass ratio.
//
// Every step runs in FP64 dual numbers (value, tangent): the leaf masses,
// the M2M shifts, every cell-to-cell interaction (the pair formula of
// pair_formula.cuh instantiated with the dual scalar), the L2L shifts and the
// evaluation.  Leaf-leaf pairs have a fixed R, so their tangent is the
// lattice kernel applied to the mass tangents.  The tangent arrays (moments,
// records, expansions) sit beside the tree's own; the values are recomputed
// alongside, so one call gives phi, g and their tangents.
#include "tangent.hpp"

#include "lattice.hpp"
#include "items.cuh"
#include "pair_formula.cuh"

namespace otfmm {

namespace {

struct Dual {
    double v, d;
    __host__ __device__ Dual() {}
    __host__ __device__ Dual(double a) : v(a), d(0.0) {}
    __host__ __device__ Dual(double a, double b) : v(a), d(b) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, fma(a.d, b.v, a.v * b.d)); }
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) {
    a.v += b.v;
    a.d += b.d;
    return a;
}
__device__ __forceinline__ Dual fma_(Dual a, Dual b, Dual c) {
    return Dual(fma(a.v, b.v, c.v), fma(a.d, b.v, fma(a.v, b.d, c.d)));
}
__device__ __forceinline__ Dual rsqrt_(Dual a) {
    const double y = otfmm::rsqrt_(a.v);
    return Dual(y, -0.5 * y * y * y * a.d);
}
__device__ __forceinline__ Dual recip(Dual a) {
    const double y = 1.0 / a.v;
    return Dual(y, -y * y * a.d);
}

constexpr int kMaxWarps = 4;

// Packed positions of symmetric tensors: rank 2 (xx xy xz yy yz zz) and
// rank 3 (xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz), indices in any order.
__host__ __device__ constexpr int sym2(int u, int v) {
    return u > v ? sym2(v, u) : (u == 0 ? v : (u == 1 ? 2 + v : 5));
}
__host__ __device__ constexpr int sym3(int u, int v, int w) {
    return u > v ? sym3(v, u, w)
                 : (v > w ? sym3(u, w, v)
                          : (u == 0 ? (v == 0 ? w : (v == 1 ? 2 + w : 5)) : (u == 1 ? (v == 1 ? 5 + w : 8) : 9)));
}

__device__ __forceinline__ Dual at(const double* v, const double* d, long long i) { return Dual(v[i], d[i]); }

// Leaf masses and their tangents; the leaf cells' expansions cleared.
__global__ void __launch_bounds__(256) k_tan_leaf(DevTree t, TanArrays a, const int* __restrict__ leaf_node,
                                                  const double* __restrict__ rho,
                                                  const double* __restrict__ rho_dot) {
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    const int L = t.node_level[node];
    const double h = t.size / (double)(8 << L);
    const double h3 = h * h * h;
    const long long N = t.n_cells;
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
        const long long cell = (long long)node * kCells + c;
        const long long o = (long long)leaf * kCells + c;
        const double m = rho[o] * h3, md = rho_dot[o] * h3;
        t.mom64[cell] = m;
        t.rec64[cell * kRec] = m;
        a.mom_d[cell] = md;
        a.rec_d[cell * kRec] = md;
#pragma unroll
        for (int r = 0; r < kLoc; r++) {
            t.loc[r * N + cell] = 0.0;
            a.loc_d[r * N + cell] = 0.0;
        }
    }
}

// M2M in dual numbers, one thread per parent cell over its 8 children (in
// parent cell units; leaf children have zero offset and higher moments):
//   M = sum m,  X = sum m pos / M,  d = pos - X,
//   M2 = sum M2_c / 4 + m d d,  M3 = sum M3_c / 8 + sym(M2_c / 4, d) + m d d d.
// A cell of zero mass keeps its geometric centre (value and tangent).
__global__ void __launch_bounds__(128) k_tan_m2m(DevTree t, TanArrays a, int first) {
    const int node = first + blockIdx.x / 4;
    const int child0 = t.node_child[node];
    if (child0 < 0) return;
    const long long N = t.n_cells;
    const int c = (blockIdx.x & 3) * 128 + threadIdx.x;
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int cn = child0 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2);
    long long cc[8];
    Dual m[8], pos[8][3];
    Dual M(0.0), X[3] = {Dual(0.0), Dual(0.0), Dual(0.0)};
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int e[3] = {q & 1, (q >> 1) & 1, q >> 2};
        cc[q] = (long long)cn * kCells + (2 * (i & 3) + e[0]) + 8 * (2 * (j & 3) + e[1]) +
                64 * (2 * (k & 3) + e[2]);
        m[q] = at(t.mom64, a.mom_d, cc[q]);
        M += m[q];
#pragma unroll
        for (int s = 0; s < 3; s++) {
            pos[q][s] = Dual(0.5) * (Dual(e[s] - 0.5) + at(t.mom64, a.mom_d, (1 + s) * N + cc[q]));
            X[s] += m[q] * pos[q][s];
        }
    }
    const Dual iM = M.v != 0.0 ? recip(M) : Dual(0.0);
#pragma unroll
    for (int s = 0; s < 3; s++) X[s] = X[s] * iM;
    Dual S2[6], S3[10];
#pragma unroll
    for (int r = 0; r < 6; r++) S2[r] = Dual(0.0);
#pragma unroll
    for (int r = 0; r < 10; r++) S3[r] = Dual(0.0);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const Dual d[3] = {pos[q][0] - X[0], pos[q][1] - X[1], pos[q][2] - X[2]};
        Dual c2[6];
#pragma unroll
        for (int r = 0; r < 6; r++) c2[r] = Dual(0.25) * at(t.mom64, a.mom_d, (4 + r) * N + cc[q]);
        const Dual mq = m[q];
        // M2 += c2 + m d d
        S2[0] += c2[0] + mq * d[0] * d[0];
        S2[1] += c2[1] + mq * d[0] * d[1];
        S2[2] += c2[2] + mq * d[0] * d[2];
        S2[3] += c2[3] + mq * d[1] * d[1];
        S2[4] += c2[4] + mq * d[1] * d[2];
        S2[5] += c2[5] + mq * d[2] * d[2];
        // M3 += M3_c / 8 + (c2_ij d_k + c2_ik d_j + c2_jk d_i) + m d d d
        const int P3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                               {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
#pragma unroll
        for (int r = 0; r < 10; r++) {
            const int u = P3[r][0], v = P3[r][1], w = P3[r][2];
            const Dual s3 = c2[sym2(u, v)] * d[w] + c2[sym2(u, w)] * d[v] + c2[sym2(v, w)] * d[u];
            S3[r] += Dual(0.125) * at(t.mom64, a.mom_d, (10 + r) * N + cc[q]) + s3 + mq * d[u] * d[v] * d[w];
        }
    }
    const long long cell = (long long)node * kCells + c;
    Dual V[kRec];
    V[0] = M;
#pragma unroll
    for (int s = 0; s < 3; s++) V[1 + s] = X[s];
#pragma unroll
    for (int r = 0; r < 6; r++) V[4 + r] = S2[r];
#pragma unroll
    for (int r = 0; r < 10; r++) V[10 + r] = S3[r];
    V[20] = S3[0] + S3[3] + S3[5];
    V[21] = S3[1] + S3[6] + S3[8];
    V[22] = S3[2] + S3[7] + S3[9];
    V[23] = S2[0] + S2[3] + S2[5];
#pragma unroll
    for (int r = 0; r < kMom; r++) {
        t.mom64[r * N + cell] = V[r].v;
        a.mom_d[r * N + cell] = V[r].d;
    }
#pragma unroll
    for (int r = 0; r < kRec; r++) {
        t.rec64[cell * kRec + r] = V[r].v;
        a.rec_d[cell * kRec + r] = V[r].d;
    }
#pragma unroll
    for (int r = 0; r < kLoc; r++) {
        t.loc[r * N + cell] = 0.0;
        a.loc_d[r * N + cell] = 0.0;
    }
}

// Source and target loads in dual numbers from the FP64 records.
__device__ __forceinline__ void head_d(const DevTree& t, const TanArrays& a, long long c, Dual& m, Dual& x,
                                       Dual& y, Dual& z) {
    const double* p = t.rec64 + c * kRec;
    const double* q = a.rec_d + c * kRec;
    m = Dual(p[0], q[0]);
    x = Dual(p[1], q[1]);
    y = Dual(p[2], q[2]);
    z = Dual(p[3], q[3]);
}
__device__ __forceinline__ void tail_d(const DevTree& t, const TanArrays& a, long long c, Dual* b2, Dual* b3,
                                       Dual* bt) {
    const double* p = t.rec64 + c * kRec;
    const double* q = a.rec_d + c * kRec;
#pragma unroll
    for (int r = 0; r < 6; r++) b2[r] = Dual(p[4 + r], q[4 + r]);
#pragma unroll
    for (int r = 0; r < 10; r++) b3[r] = Dual(p[10 + r], q[10 + r]);
#pragma unroll
    for (int r = 0; r < 4; r++) bt[r] = Dual(p[20 + r], q[20 + r]);
}

__device__ __forceinline__ void add_d(const DevTree& t, const TanArrays& a, long long i, Dual v, double s) {
    atomicAdd(t.loc + i, s * v.v);
    atomicAdd(a.loc_d + i, s * v.d);
}

// One work item of the forward plan in dual numbers (the generic loop of the
// FP64 general kernel).
template <bool FULL, bool AM>
__device__ __forceinline__ void tan_item(const DevTree& t, const TanArrays& a, const DevPlan& p,
                                         const int4 it, const int lane, const int* s_nb, const int* s_lf,
                                         const LevelScales& sc) {
    const int node = it.x;
    const int L = item_level(it);
    int i, j, k;
    item_cell(p, it, lane, i, j, k);
    const long long N = t.n_cells;
    const long long cell = (long long)node * kCells + i + 8 * j + 64 * k;
    Dual ma, dax, day, daz;
    head_d(t, a, cell, ma, dax, day, daz);
    Acc<Dual> A;
    acc_zero(A);
    auto pair = [&](Dual x, Dual y, Dual z, Dual m, long long src, bool sleaf) {
        if (sleaf) {
            m2l_pair<Dual, FULL, false, AM>(x, y, z, m, nullptr, nullptr, nullptr, A);
        } else {
            Dual b2[6], b3[10], bt[4];
            tail_d(t, a, src, b2, b3, bt);
            m2l_pair<Dual, FULL, true, AM>(x, y, z, m, b2, b3, bt, A);
        }
    };
    // A pair through stencil entry ent with a source of kind 2 (leaf) or 3
    // (interior); with multi, leaf sources take the multipole formula with
    // zero moments (the same sums, one pass for the warp).
    auto pair_at = [&](int kind, bool multi, long long src, int ent) {
        Dual m, bx, by, bz;
        head_d(t, a, src, m, bx, by, bz);
        const double2 o0 = __ldg(p.off64 + 2 * ent), o1 = __ldg(p.off64 + 2 * ent + 1);
        const Dual x = (dax - bx) - Dual(o0.x), y = (day - by) - Dual(o0.y), z = (daz - bz) - Dual(o1.x);
        if (!multi) {
            m2l_pair<Dual, FULL, false, AM>(x, y, z, m, nullptr, nullptr, nullptr, A);
            return;
        }
        Dual b2[6], b3[10], bt[4];
        if (kind == 3) {
            tail_d(t, a, src, b2, b3, bt);
        } else {
#pragma unroll
            for (int r = 0; r < 6; r++) b2[r] = Dual(0.0);
#pragma unroll
            for (int r = 0; r < 10; r++) b3[r] = Dual(0.0);
#pragma unroll
            for (int r = 0; r < 4; r++) bt[r] = Dual(0.0);
        }
        m2l_pair<Dual, FULL, true, AM>(x, y, z, m, b2, b3, bt, A);
    };
    if (FULL && item_list(it) == kRootList) {
        const int root = it.x;
#pragma unroll 1
        for (int s = it.z; s < it.w; s++) {
            const int sx = s & 7, sy = (s >> 3) & 7, sz = s >> 6;
            const int dx = sx - i, dy = sy - j, dz = sz - k;
            if (dx * dx + dy * dy + dz * dz <= p.near_d2) continue;
            const long long src = (long long)root * kCells + s;
            Dual m, bx, by, bz;
            head_d(t, a, src, m, bx, by, bz);
            pair((dax - bx) - Dual((double)dx), (day - by) - Dual((double)dy), (daz - bz) - Dual((double)dz),
                 m, src, false);
        }
    } else if (item_list(it) == kGroupList) {
        // grouped item: every lane walks its own list (as in the FP64 kernel)
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
            // pair kinds as in the FP64 kernel: 0 none, 1 point masses of a
            // leaf root, 2 leaf source, 3 interior source
            int kind = 0;
            if (nb >= 0) {
                if (!FULL && sleaf) kind = L > 0 ? 0 : 1;
                else if (!(FULL && !sleaf && entry_near(e))) kind = sleaf ? 2 : 3;
            }
            const bool multi = __any_sync(0xffffffffu, kind == 3);
            if (kind == 0) continue;
            const long long src = (long long)nb * kCells + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
            if (kind == 1) {
                // two point masses on the lattice (a leaf root): fixed coefficients
                const double2 k0 = __ldg(p.tab64 + 2 * (base + q)), k1 = __ldg(p.tab64 + 2 * (base + q) + 1);
                const Dual m = at(t.mom64, a.mom_d, src);
                A.L0 = fma_(m, Dual(k0.x), A.L0);
                A.L1[0] = fma_(m, Dual(k0.y), A.L1[0]);
                A.L1[1] = fma_(m, Dual(k1.x), A.L1[1]);
                A.L1[2] = fma_(m, Dual(k1.y), A.L1[2]);
                continue;
            }
            pair_at(kind, multi, src, base + q);
        }
    }
    const double* sl = sc.s64[L];
    add_d(t, a, cell, A.L0, sl[0]);
#pragma unroll
    for (int r = 0; r < 3; r++) add_d(t, a, (1 + r) * N + cell, A.L1[r], sl[1]);
    if (FULL) {
        finish_acc(A);
#pragma unroll
        for (int r = 0; r < 6; r++) add_d(t, a, (4 + r) * N + cell, A.L2[r], kAccL2 * sl[2]);
#pragma unroll
        for (int r = 0; r < 10; r++) add_d(t, a, (10 + r) * N + cell, A.L3[r], kAccL3 * sl[3]);
    }
    if (AM) {
        Dual P[3] = {Dual(0.0), Dual(0.0), Dual(0.0)};
        if (FULL) {
            // the target's octupole per unit mass (zero for a target of zero mass)
            Dual a3[10], ta[3];
            const Dual r = ma.v != 0.0 ? recip(ma) : Dual(0.0);
            const double* pv = t.rec64 + cell * kRec;
            const double* pd = a.rec_d + cell * kRec;
#pragma unroll
            for (int q = 0; q < 10; q++) a3[q] = r * Dual(pv[10 + q], pd[10 + q]);
#pragma unroll
            for (int q = 0; q < 3; q++) ta[q] = r * Dual(pv[20 + q], pd[20 + q]);
            correction_target(A, a3, ta, P);
        }
#pragma unroll
        for (int r = 0; r < 3; r++) add_d(t, a, (20 + r) * N + cell, A.S[r] - P[r], kAccCor * sl[4]);
    }
}

__global__ void __launch_bounds__(128) k_tan_interact(DevTree t, TanArrays a, DevPlan p, LevelScales sc, int am) {
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
            if (am) tan_item<true, true>(t, a, p, it, lane, s_nb[w], s_lf[w], sc);
            else tan_item<true, false>(t, a, p, it, lane, s_nb[w], s_lf[w], sc);
        } else {
            if (am) tan_item<false, true>(t, a, p, it, lane, s_nb[w], s_lf[w], sc);
            else tan_item<false, false>(t, a, p, it, lane, s_nb[w], s_lf[w], sc);
        }
        __syncwarp();
    }
}

// E += exact degree-3 shift of the parent's expansion P by delta (physical
// units) and the parent's correction acceleration:
//   L0 += P0 + P1.d + d.P2.d / 2 + P3:ddd / 6,  L1 += P1 + P2 d + P3:dd / 2,
//   L2 += P2 + P3 . d,  L3 += P3,  a_c += a_c(parent).
__device__ __forceinline__ void shift_add(Dual* E, const Dual* P, const Dual* dl) {
    const Dual* L2 = P + 4;
    const Dual* L3 = P + 10;
    // T2 = P3 . d (packed rank 2), T1 = P2 d + T2 d / 2, T0 = P1.d + d.P2.d / 2 + d.T2.d / 6
    Dual T2[6];
#pragma unroll
    for (int r = 0; r < 6; r++) T2[r] = Dual(0.0);
#pragma unroll
    for (int u = 0; u < 3; u++)
#pragma unroll
        for (int v = u; v < 3; v++)
#pragma unroll
            for (int w = 0; w < 3; w++) T2[sym2(u, v)] += L3[sym3(u, v, w)] * dl[w];
    Dual P2d[3], T2d[3];
#pragma unroll
    for (int u = 0; u < 3; u++) {
        P2d[u] = L2[sym2(u, 0)] * dl[0] + L2[sym2(u, 1)] * dl[1] + L2[sym2(u, 2)] * dl[2];
        T2d[u] = T2[sym2(u, 0)] * dl[0] + T2[sym2(u, 1)] * dl[1] + T2[sym2(u, 2)] * dl[2];
    }
    Dual s0 = P[0];
#pragma unroll
    for (int u = 0; u < 3; u++)
        s0 += dl[u] * (P[1 + u] + Dual(0.5) * P2d[u] + Dual(1.0 / 6.0) * T2d[u]);
    E[0] += s0;
#pragma unroll
    for (int u = 0; u < 3; u++) E[1 + u] += P[1 + u] + P2d[u] + Dual(0.5) * T2d[u];
#pragma unroll
    for (int r = 0; r < 6; r++) E[4 + r] += L2[r] + T2[r];
#pragma unroll
    for (int r = 0; r < 10; r++) E[10 + r] += L3[r];
#pragma unroll
    for (int r = 0; r < 3; r++) E[20 + r] += P[20 + r];
}

// Downward pass of one level in dual numbers, one thread per cell: an
// interior cell below the root adds its parent's shifted expansion (in
// place); a leaf cell adds it to its own terms and is evaluated.
__global__ void __launch_bounds__(128) k_tan_down(DevTree t, TanArrays a, int first, const double* __restrict__ rho,
                                                  const double* __restrict__ rho_dot, double* __restrict__ phi,
                                                  double* __restrict__ g, double* __restrict__ phi_dot,
                                                  double* __restrict__ g_dot, double G, int self_term) {
    const int node = first + blockIdx.x / 4;
    const int c = (blockIdx.x & 3) * 128 + threadIdx.x;
    const int L = t.node_level[node];
    const int parent = t.node_parent[node];
    const int leaf = t.node_leaf[node];
    if (leaf < 0 && parent < 0) return;  // the interior root: nothing to add
    const long long N = t.n_cells;
    const double h = t.size / (double)(8 << L);
    const int* xyz = t.node_xyz + 3 * node;
    const int ci[3] = {c & 7, (c >> 3) & 7, c >> 6};
    const long long cell = (long long)node * kCells + c;
    Dual E[kLoc];
#pragma unroll
    for (int r = 0; r < kLoc; r++)
        E[r] = (leaf < 0 || r < 4 || r >= 20) ? at(t.loc, a.loc_d, r * N + cell) : Dual(0.0);
    if (parent >= 0) {
        int pl = 0, off[3];
#pragma unroll
        for (int s = 0; s < 3; s++) {
            const int gc = 8 * xyz[s] + ci[s];
            off[s] = gc & 1;
            pl += ((gc >> 1) & 7) << (3 * s);
        }
        const long long pcell = (long long)parent * kCells + pl;
        Dual P[kLoc];
#pragma unroll
        for (int r = 0; r < kLoc; r++) P[r] = at(t.loc, a.loc_d, r * N + pcell);
        // delta = X_cell - X_parent = h ((off - 1/2) + dX_cell - 2 dX_parent)
        Dual dl[3];
#pragma unroll
        for (int s = 0; s < 3; s++)
            dl[s] = Dual(h) * ((Dual(off[s] - 0.5) + at(t.mom64, a.mom_d, (1 + s) * N + cell)) -
                               Dual(2.0) * at(t.mom64, a.mom_d, (1 + s) * N + pcell));
        shift_add(E, P, dl);
    }
    if (leaf < 0) {
#pragma unroll
        for (int r = 0; r < kLoc; r++) {
            t.loc[r * N + cell] = E[r].v;
            a.loc_d[r * N + cell] = E[r].d;
        }
        return;
    }
    const long long o = (long long)leaf * kCells + c;
    Dual p = E[0];
    if (self_term) {
        const double cs = -G * h * h * 3.0 * (log(2.0 + sqrt(3.0)) - 3.14159265358979323846 / 6.0);
        p += Dual(cs * rho[o], cs * rho_dot[o]);
    }
    if (phi) phi[o] = p.v;
    phi_dot[o] = p.d;
#pragma unroll
    for (int s = 0; s < 3; s++) {
        const Dual gv = E[20 + s] - E[1 + s];
        if (g) g[((long long)leaf * 3 + s) * kCells + c] = gv.v;
        g_dot[((long long)leaf * 3 + s) * kCells + c] = gv.d;
    }
}

}  // namespace

void launch_tangent(const DevTree& t, const TanArrays& a, const int* leaf_node, const DevPlan& p,
                    const DevLattice& lp, const int* level_first, int n_levels, const double* rho,
                    const double* rho_dot, double* phi, double* g, double* phi_dot, double* g_dot, double G,
                    int am, int self_term, int ctas, cudaStream_t s) {
    k_tan_leaf<<<t.n_leaf, 256, 0, s>>>(t, a, leaf_node, rho, rho_dot);
    for (int L = n_levels - 2; L >= 0; L--) {
        const int count = level_first[L + 1] - level_first[L];
        if (count > 0) k_tan_m2m<<<count * 4, 128, 0, s>>>(t, a, level_first[L]);
    }
    const LevelScales sc = level_scales(t.inv_side8, G);
    // leaf-leaf pairs: values from the masses, tangents from the mass
    // tangents (R is fixed on the lattice), on the same stream
    launch_lattice(t, p, lp, kPrecFP64, G, 0, s);
    DevTree td = t;
    td.mom64 = a.mom_d;
    td.loc = a.loc_d;
    DevLattice lp2 = lp;
    lp2.counter = lp.counter + 1;  // the second pair of node counters
    launch_lattice(td, p, lp2, kPrecFP64, G, 0, s);
    DevPlan pg = p;  // the grouped items where the plan has them
    if (p.items_grp) {
        pg.items = p.items_grp;
        pg.n_items = p.n_items_grp;
    }
    k_tan_interact<<<ctas, 128, 0, s>>>(t, a, pg, sc, am);
    for (int L = 0; L < n_levels; L++) {
        const int count = level_first[L + 1] - level_first[L];
        if (count > 0)
            k_tan_down<<<count * 4, 128, 0, s>>>(t, a, level_first[L], rho, rho_dot, phi, g, phi_dot, g_dot, G,
                                                 self_term);
    }
}

}  // namespace otfmm
