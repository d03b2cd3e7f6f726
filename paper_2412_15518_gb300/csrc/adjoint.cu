// Hand-written adjoint of the FMM gravity solve on GB300 (FP64).
//
// For J = sum_c (w1_c phi_c + w2_c . g_c) the reverse sweep runs the forward
// steps backwards:
//   seeds      leaf cells: E0 = w1, E1 = -w2, a = w2 (phi = L0, g = -L1 + a_c)
//   L2L^T      per interior cell, gathered over its 8 children, bottom-up:
//              E_parent = sum shift^T(E_child, delta), a_parent = sum a_child,
//              delta-bar to the children's and the parent's centre of mass
//   M2L^T      every directed pair reversed once: a pair with an interior
//              target in that target's pass (its centre of mass and the
//              correction's mass ratio gathered, the source's moment and
//              centre-of-mass adjoints sent by atomics), a pair with a leaf
//              target in the source's pass; leaf-leaf pairs use the lattice
//              table transposed; one persistent launch over all levels
//   M2M^T      per interior cell, top-down: adjoints of the 8 children's
//              moments and centres of mass
//   density    drho = h^3 dJ/dm (+ the self term)
// Adjoint arrays (physical units, FP64, structure of arrays):
//   locbar [23][cells]  E0, E1(3), E2(6), E3(10) symmetric adjoints of the
//                       expansion, and the adjoint of a_c (3)
//   mombar [20][cells]  dJ/dm, dJ/dX(3), dJ/dM2(6), dJ/dM3(10) (symmetric)
//   a4     [15][cells]  the interior targets' quartic sums sum_B m_B f4 R^4
//                       (cell units), added by the forward part's general
//                       kernel (p.a4_out) and read here once per target
#include "adjoint.hpp"
#include "adjoint_pair.cuh"
#include "items.cuh"

namespace otfmm {

namespace {

__host__ __device__ inline double cube_self_c() {
    return 3.0 * (log(2.0 + sqrt(3.0)) - 3.14159265358979323846 / 6.0);
}

__global__ void __launch_bounds__(256) k_adj_seed(DevTree t, const int* __restrict__ leaf_node,
                                                  const double* __restrict__ w1,
                                                  const double* __restrict__ w2, double* locbar) {
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    const long long N = t.n_cells;
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
        const long long cell = (long long)node * kCells + c;
        locbar[cell] = w1[(long long)leaf * kCells + c];
        for (int a = 0; a < 3; a++) {
            const double wg = w2[((long long)leaf * 3 + a) * kCells + c];
            locbar[(1 + a) * N + cell] = -wg;
            locbar[(20 + a) * N + cell] = wg;
        }
        for (int r = 4; r < 20; r++) locbar[r * N + cell] = 0.0;
    }
}

// Butterfly step of a reduce-scatter over lanes q and q ^ mask: a lane keeps
// the component of each pair (lo, hi) on its own side of the mask bit, adds
// its partner's copy of it, and hands over the other one.
__device__ __forceinline__ double keep_add(bool upper, double lo, double hi, int mask) {
    const double keep = upper ? hi : lo;
    const double give = upper ? lo : hi;
    return keep + __shfl_xor_sync(0xffffffffu, give, mask);
}

// Sum over the 8 lanes of a parent cell of 32 values: lane q ends with the
// sums of components q, q + 8, q + 16 and q + 24 (out[0..3]).
__device__ __forceinline__ void reduce_scatter8(const double* V, int q, double* out) {
    const bool u4 = q & 4, u2 = q & 2, u1 = q & 1;
    double R16[16], R8[8];
#pragma unroll
    for (int h = 0; h < 16; h++) {
        const int lo = (h & 3) | ((h & 12) << 1);  // components with bit 2 clear
        R16[h] = keep_add(u4, V[lo], V[lo | 4], 4);
    }
#pragma unroll
    for (int g = 0; g < 8; g++) {
        const int lo = (g & 1) | ((g & 6) << 1);
        R8[g] = keep_add(u2, R16[lo], R16[lo | 2], 2);
    }
#pragma unroll
    for (int f = 0; f < 4; f++) out[f] = keep_add(u1, R8[2 * f], R8[2 * f + 1], 1);
}

__device__ __forceinline__ double sum8(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}

// L2L reverse at parent level: 8 lanes per parent cell, one per child (one
// warp = 4 parent cells, 128 blocks per node, so even the single level-0 node
// spreads over 128 SMs).  The forward shift by d = X_child - X_parent is
//   C0 = L0 + L1.d + d.L2.d / 2 + L3:ddd / 6,  C1 = L1 + L2 d + L3:dd / 2,
//   C2 = L2 + L3 d,  C3 = L3,
// so with the child's adjoints C the parent's adjoints E gather
//   E0 += C0,  E1 += C0 d + C1,  E2 += C0 dd / 2 + sym(C1 d) + C2,
//   E3 += C0 ddd / 6 + sym(C1 dd) / 6 + sym(C2 d) / 3 + C3,
// and d gets dbar = C0 (L1 + L2 d + L3:dd / 2) + L2 C1 + L3:sym(C1 d) + L3:C2,
// added to the child's centre of mass and subtracted from the parent's.  The
// parent's sums over its children are a reduce-scatter over the 8 lanes.
__global__ void __launch_bounds__(32) k_l2l_reverse(DevTree t, int first, double* locbar,
                                                    double* mombar) {
    const int node = first + (blockIdx.x >> 7);
    const int child0 = t.node_child[node];
    if (child0 < 0) return;
    const long long N = t.n_cells;
    const int L = t.node_level[node];
    const double hc = t.size / (double)(16 << L);  // child cell side
    const int c = ((blockIdx.x & 127) << 2) + (threadIdx.x >> 3);  // parent cell in the node
    const int q = threadIdx.x & 7;                                  // child octant
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const long long pcell = (long long)node * kCells + c;
    double P[20];
#pragma unroll
    for (int r = 0; r < 20; r++) P[r] = t.loc[r * N + pcell];
    const double* L2 = P + 4;
    const double* L3 = P + 10;
    const double pd[3] = {t.mom64[N + pcell], t.mom64[2 * N + pcell], t.mom64[3 * N + pcell]};
    const int cn = child0 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2);
    const int a = q & 1, b = (q >> 1) & 1, e = q >> 2;
    const long long cc = (long long)cn * kCells + (2 * (i & 3) + a) + 8 * (2 * (j & 3) + b) +
                         64 * (2 * (k & 3) + e);
    const double d[3] = {hc * ((a - 0.5) + t.mom64[N + cc] - 2.0 * pd[0]),
                         hc * ((b - 0.5) + t.mom64[2 * N + cc] - 2.0 * pd[1]),
                         hc * ((e - 0.5) + t.mom64[3 * N + cc] - 2.0 * pd[2])};
    double C[20];
#pragma unroll
    for (int r = 0; r < 20; r++) C[r] = locbar[r * N + cc];
    const double C0 = C[0];
    const double* C1 = C + 1;
    const double* C2 = C + 4;
    RMono<double> md;
    r_mono(d[0], d[1], d[2], md);
    // this child's part of the parent's sums: V[0..19] = E, V[20..22] = a,
    // V[23..25] = the parent's centre-of-mass adjoint; V[26..31] unused
    double V[32];
#pragma unroll
    for (int r = 0; r < 32; r++) V[r] = 0.0;
    double* E = V;
    // E0, E1
    E[0] = C0;
#pragma unroll
    for (int s = 0; s < 3; s++) E[1 + s] = C0 * d[s] + C1[s];
    // E2 = C0 dd / 2 + sym(C1 d) + C2  (sym(C1 d)_uv = (C1_u d_v + C1_v d_u) / 2)
    const double h0 = 0.5 * C0;
    E[4] = h0 * md.xx + C1[0] * d[0] + C2[0];
    E[5] = h0 * md.xy + 0.5 * (C1[0] * d[1] + C1[1] * d[0]) + C2[1];
    E[6] = h0 * md.xz + 0.5 * (C1[0] * d[2] + C1[2] * d[0]) + C2[2];
    E[7] = h0 * md.yy + C1[1] * d[1] + C2[3];
    E[8] = h0 * md.yz + 0.5 * (C1[1] * d[2] + C1[2] * d[1]) + C2[4];
    E[9] = h0 * md.zz + C1[2] * d[2] + C2[5];
    // E3 = C0 ddd / 6 + (C1 dd)_sym / 6 + (C2 d)_sym / 3 + C3
    add_rank3(E + 10, md, C1, C0 / 6.0, 1.0 / 6.0, 0.0, 0.0);
    const double t3 = 1.0 / 3.0;
    E[10] += t3 * (3.0 * C2[0] * d[0]) + C[10];
    E[11] += t3 * (C2[0] * d[1] + 2.0 * C2[1] * d[0]) + C[11];
    E[12] += t3 * (C2[0] * d[2] + 2.0 * C2[2] * d[0]) + C[12];
    E[13] += t3 * (2.0 * C2[1] * d[1] + C2[3] * d[0]) + C[13];
    E[14] += t3 * (C2[1] * d[2] + C2[2] * d[1] + C2[4] * d[0]) + C[14];
    E[15] += t3 * (2.0 * C2[2] * d[2] + C2[5] * d[0]) + C[15];
    E[16] += t3 * (3.0 * C2[3] * d[1]) + C[16];
    E[17] += t3 * (C2[3] * d[2] + 2.0 * C2[4] * d[1]) + C[17];
    E[18] += t3 * (2.0 * C2[4] * d[2] + C2[5] * d[1]) + C[18];
    E[19] += t3 * (3.0 * C2[5] * d[2]) + C[19];
#pragma unroll
    for (int s = 0; s < 3; s++) V[20 + s] = locbar[(20 + s) * N + cc];
    // dbar = C0 (L1 + L2 d + L3:dd / 2) + L2 C1 + L3:sym(C1 d) + L3:C2, added
    // to the child's centre of mass and subtracted from the parent's
    double L2d[3], L3dd[3], L2C1[3], L3C1d[3], L3C2[3];
    sym2_vec(L2, d, L2d);
    sym3_contract(L3, md.xx, md.yy, md.zz, md.xy2, md.xz2, md.yz2, L3dd);
    sym2_vec(L2, C1, L2C1);
    sym3_contract(L3, C1[0] * d[0], C1[1] * d[1], C1[2] * d[2], C1[0] * d[1] + C1[1] * d[0],
                  C1[0] * d[2] + C1[2] * d[0], C1[1] * d[2] + C1[2] * d[1], L3C1d);
    sym3_contract(L3, C2[0], C2[3], C2[5], 2.0 * C2[1], 2.0 * C2[2], 2.0 * C2[4], L3C2);
#pragma unroll
    for (int s = 0; s < 3; s++) {
        const double db = C0 * (P[1 + s] + L2d[s] + 0.5 * L3dd[s]) + L2C1[s] + L3C1d[s] + L3C2[s];
        mombar[(1 + s) * N + cc] += db;  // this lane's child only
        V[23 + s] = -db;
    }
    // the parent's sums: component r = q + 8 f of the 32; r < 23 is
    // locbar[r], 23..25 the parent's centre-of-mass adjoint
    double S[4];
    reduce_scatter8(V, q, S);
#pragma unroll
    for (int f = 0; f < 4; f++) {
        const int r = q + 8 * f;
        if (r < 23) locbar[r * N + pcell] = S[f];
        else if (r < 26) mombar[(r - 22) * N + pcell] += S[f];
    }
}

// Grouped reverse items (interior cells of level >= 1): moves q, this lane's
// position in the list of its own parity class, to its next partner in
// [q, qend) that the pass reverses -- pass 1 a leaf partner (this cell is the
// source of the leaf's expansion), pass 2 a leaf partner or a far interior
// one (this cell is the target) -- and returns 2 for a leaf partner, 3 for an
// interior one, 0 when none is left; e = the entry, nb/lc = the partner's
// node and node-local cell.
template <int PASS>
__device__ __forceinline__ int next_partner(const DevPlan& p, const int* s_nb, const int* s_lf, int base,
                                            int qend, int i, int j, int k, int& q, int& e, int& nb,
                                            int& lc) {
    for (; q < qend; q++) {
        const int en = __ldg(p.entries + base + q);
        const int sx = i + entry_dx(en), sy = j + entry_dy(en), sz = k + entry_dz(en);
        const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
        const int n = s_nb[slot];
        if (n < 0) continue;
        const bool pleaf = s_lf[slot] != 0;
        if (PASS == 1 ? !pleaf : (!pleaf && entry_near(en))) continue;
        e = en;
        nb = n;
        lc = (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
        return pleaf ? 2 : 3;
    }
    return 0;
}

// What a pass-2 target holds for all its pairs and reads once or twice per
// pair: its E2, E3 and octupole, and its partner-independent parts.  Kept in
// shared memory, one record per lane (37 doubles: consecutive lanes' records
// start 2 banks apart, so a warp's access is conflict-free), which leaves the
// registers to the pair itself.
struct RevLane {
    double e2[6], e3[10], m3[10];
    RevTarget<double> tg;
};
static_assert(sizeof(RevLane) == 37 * sizeof(double), "odd record length in doubles");

// M2L / near-pair reverse: persistent over the reverse work items.  A
// parity-class item runs both passes for its 32 cells; a grouped item (32
// interior cells of one node sorted by their numbers of partners) runs one,
// every lane walking its own list.
__global__ void __launch_bounds__(128) k_m2l_reverse(DevTree t, DevPlan p, const double* locbar,
                                                     double* mombar, double G, int am) {
    __shared__ int s_nb[4][28];
    __shared__ int s_lf[4][28];
    __shared__ RevLane s_rl[4][32];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    RevLane& rl = s_rl[w][lane];
    const long long N = t.n_cells;
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
        const int node = it.x;
        const bool cleaf = t.node_leaf[node] >= 0;
        const int L = item_level(it);
        const bool grp = item_list(it) == kGroupList;
        // an interior root's items range over its own 512 cells as partners
        // (all interior: pass 2 only)
        const bool rootc = item_list(it) == kRootList;
        const int passes = grp ? (it.y >> 16) & 3 : (rootc ? 2 : 3);  // bit 0: pass 1, bit 1: pass 2
        int i, j, k;
        item_cell(p, it, lane, i, j, k);
        const long long cell = (long long)node * kCells + i + 8 * j + 64 * k;
        // the list and its range: a grouped item's lane walks its own parity list
        int base, q0, q1;
        if (grp) {
            const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
            base = __ldg(p.list_first + par);
            q0 = it.z & 0xffff;
            q1 = min(it.z >> 16, __ldg(p.list_len + par));
        } else {
            base = rootc ? 0 : p.list_first[item_list(it)];
            q0 = it.z;
            q1 = it.w;
        }
        // The pairs run in cell units (R, M2, M3 of this level) with the
        // adjoints pre-scaled by -G h^-(n+1) (E_n) and -(G/6) h^-2 (a); their
        // moment and centre-of-mass adjoints come out physical through the
        // factors h^-2, h^-3 and h^-1 (m2l_pair_reverse).
        const double h = t.size / (double)(8 << L);
        const double hi = 1.0 / h, hi2 = hi * hi, hi3 = hi2 * hi;
        const double sE0 = -G * hi, sE1 = sE0 * hi, sE2 = sE1 * hi, sE3 = sE2 * hi;
        const double sA = (-G / 6.0) * hi2;
        // own moments (cell units) and own expansion adjoints
        const double mC = t.mom64[cell];
        const double dC[3] = {t.mom64[N + cell], t.mom64[2 * N + cell], t.mom64[3 * N + cell]};
        double M2C[6], M3C[10], btC[4];  // btC: M3's trace vector, trace of M2
        if (!cleaf) {
#pragma unroll
            for (int r = 0; r < 6; r++) M2C[r] = t.mom64[(4 + r) * N + cell];
#pragma unroll
            for (int r = 0; r < 10; r++) M3C[r] = t.mom64[(10 + r) * N + cell];
        } else {
#pragma unroll
            for (int r = 0; r < 6; r++) M2C[r] = 0.0;
#pragma unroll
            for (int r = 0; r < 10; r++) M3C[r] = 0.0;
        }
        sym3_trace(M3C, btC);
        btC[3] = M2C[0] + M2C[3] + M2C[5];
        PairAdjOut acc;
        adj_zero(acc);
        double lat0 = 0.0, lat1 = 0.0;   // lattice pairs: dJ/dm of this leaf cell (h, h^2 parts)
        // Two passes over the partners, each holding only what its role needs;
        // every directed pair is reversed once.  Pass 1: this cell as the
        // source of a leaf partner's expansion (R = X_P - X_C), and the
        // transposed lattice pairs of a leaf cell.  A pair with an interior
        // target is reversed whole in that target's pass 2, which sends the
        // source-side adjoints here with atomics.
        auto rev1 = [&](int e, long long pc) {
            const double R[3] = {(double)entry_dx(e) + t.mom64[N + pc] - dC[0],
                                 (double)entry_dy(e) + t.mom64[2 * N + pc] - dC[1],
                                 (double)entry_dz(e) + t.mom64[3 * N + pc] - dC[2]};
            // a leaf partner: no octupole, and only its L0/L1 adjoints exist
            const double e0 = sE0 * locbar[pc];
            double e1[3], aP[3];
#pragma unroll
            for (int r = 0; r < 3; r++) {
                e1[r] = sE1 * locbar[(1 + r) * N + pc];
                aP[r] = sA * locbar[(20 + r) * N + pc];
            }
            RevTarget<double> tg;
            reverse_target_prep<false>(e0, (const double*)nullptr, (const double*)nullptr, false, 0.0,
                                       (const double*)nullptr, aP, tg);
            // the R-gradient of this pair moves this cell's centre of mass (a
            // leaf partner's centre is fixed): R = X_P - X_C
            m2l_pair_reverse<true, false, false, double>(R, mC, M2C, M3C, btC, !cleaf, false, 0.0, M3C, e0, e1,
                                                         nullptr, nullptr, tg, am, aP, !cleaf, hi2, hi3, -hi,
                                                         acc.R, acc);
        };
        if (passes & 1) {
            if (grp) {
#pragma unroll 1
                for (int q = q0;;) {
                    int e = 0, nb = 0, lc = 0;
                    const int kind = next_partner<1>(p, s_nb[w], s_lf[w], base, q1, i, j, k, q, e, nb, lc);
                    if (!__any_sync(0xffffffffu, kind != 0)) break;
                    if (kind != 0) rev1(e, (long long)nb * kCells + lc);
                    q++;
                }
            } else {
#pragma unroll 1
                for (int q = q0; q < q1; q++) {
                    const int e = __ldg(p.entries + base + q);
                    const int sx = i + entry_dx(e), sy = j + entry_dy(e), sz = k + entry_dz(e);
                    const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
                    const int nb = s_nb[w][slot];
                    if (nb < 0) continue;
                    const bool pleaf = s_lf[w][slot] != 0;
                    const long long pc = (long long)nb * kCells + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7);
                    if (cleaf && pleaf) {
                        // transposed lattice pair: this cell is the source of P's point-mass pair
                        const double2 t0 = __ldg(p.tab64 + 2 * (base + q)), t1 = __ldg(p.tab64 + 2 * (base + q) + 1);
                        lat0 = fma(locbar[pc], t0.x, lat0);
                        lat1 = fma(locbar[N + pc], t0.y,
                                   fma(locbar[2 * N + pc], t1.x, fma(locbar[3 * N + pc], t1.y, lat1)));
                        continue;
                    }
                    if (!pleaf) continue;  // an interior target: its own pass 2
                    rev1(e, pc);
                }
            }
            // this cell's source-side adjoints of pass 1; acc's source fields
            // then carry one pair's partner adjoints at a time in pass 2
            atomicAdd(mombar + cell, acc.mB - G * (lat0 * hi - lat1 * hi2));
            acc.mB = 0.0;
            if (!cleaf) {
#pragma unroll
                for (int r = 0; r < 6; r++) {
                    atomicAdd(mombar + (4 + r) * N + cell, acc.M2B[r]);
                    acc.M2B[r] = 0.0;
                }
#pragma unroll
                for (int r = 0; r < 10; r++) {
                    atomicAdd(mombar + (10 + r) * N + cell, acc.M3B[r]);
                    acc.M3B[r] = 0.0;
                }
            }
        }
        // Pass 2 (interior cells): this cell as the target of its partners
        // (R = X_C - X_P), each pair reversed whole: the correction's mass
        // ratio and the pair's R-gradient for this cell, the partner's
        // source-side adjoints and its part of the R-gradient by atomics.
        if (!cleaf && (passes & 2)) {
            double EC[4], aC[3];
#pragma unroll
            for (int r = 0; r < 4; r++) EC[r] = (r == 0 ? sE0 : sE1) * locbar[r * N + cell];
#pragma unroll
            for (int r = 0; r < 6; r++) rl.e2[r] = sE2 * locbar[(4 + r) * N + cell];
#pragma unroll
            for (int r = 0; r < 10; r++) {
                rl.e3[r] = sE3 * locbar[(10 + r) * N + cell];
                rl.m3[r] = M3C[r];
            }
#pragma unroll
            for (int r = 0; r < 3; r++) aC[r] = sA * locbar[(20 + r) * N + cell];
            // the correction's mass-ratio term (a target of non-zero mass)
            const bool useA = am && mC != 0.0;
            const double iA = useA ? 1.0 / mC : 0.0;
            reverse_target_prep<true>(EC[0], rl.e2, rl.e3, useA, iA, rl.m3, aC, rl.tg);
            auto rev2 = [&](int dx, int dy, int dz, bool pleaf, long long pc) {
                // the partner's record: m, its centre-of-mass offset, and for
                // an interior partner M2, M3 and their traces (16-byte loads)
                const double2* pr = reinterpret_cast<const double2*>(t.rec64 + pc * kRec);
                const double2 h0 = __ldg(pr), h1 = __ldg(pr + 1);
                const double mP = h0.x;
                const double Rn[3] = {dC[0] - (double)dx - h0.y, dC[1] - (double)dy - h1.x,
                                      dC[2] - (double)dz - h1.y};
                double V[20];
#pragma unroll
                for (int r = 0; r < 10; r++) {
                    const double2 v = pleaf ? make_double2(0.0, 0.0) : __ldg(pr + 2 + r);
                    V[2 * r] = v.x;
                    V[2 * r + 1] = v.y;
                }
                const double* M2P = V;
                const double* M3P = V + 6;
                const double* btP = V + 16;
                double gR[3] = {0.0, 0.0, 0.0};
                m2l_pair_reverse<true, true, true>(Rn, mP, M2P, M3P, btP, !pleaf, useA, iA, rl.m3, EC[0], EC + 1,
                                                   rl.e2, rl.e3, rl.tg, am, aC, true, hi2, hi3, hi, gR, acc);
                // the partner's source-side adjoints of this pair
                atomicAdd(mombar + pc, acc.mB);
                acc.mB = 0.0;
                if (!pleaf) {
#pragma unroll
                    for (int r = 0; r < 6; r++) {
                        atomicAdd(mombar + (4 + r) * N + pc, acc.M2B[r]);
                        acc.M2B[r] = 0.0;
                    }
#pragma unroll
                    for (int r = 0; r < 10; r++) {
                        atomicAdd(mombar + (10 + r) * N + pc, acc.M3B[r]);
                        acc.M3B[r] = 0.0;
                    }
                }
                // dJ/dR moves both centres of mass: + this cell's, - an interior
                // partner's (a leaf's centre is fixed)
#pragma unroll
                for (int s = 0; s < 3; s++) acc.R[s] += gR[s];
                if (!pleaf) {
#pragma unroll
                    for (int s = 0; s < 3; s++) atomicAdd(mombar + (1 + s) * N + pc, -gR[s]);
                }
            };
            if (rootc) {
                // the same partner cell for every lane (a broadcast load); a
                // pair is far iff |d|^2 > near_d2 (near ones descend)
#pragma unroll 1
                for (int sc = q0; sc < q1; sc++) {
                    const int dx = (sc & 7) - i, dy = ((sc >> 3) & 7) - j, dz = (sc >> 6) - k;
                    if (dx * dx + dy * dy + dz * dz <= p.near_d2) continue;
                    rev2(dx, dy, dz, false, (long long)node * kCells + sc);
                }
            } else if (grp) {
#pragma unroll 1
                for (int q = q0;;) {
                    int e = 0, nb = 0, lc = 0;
                    const int kind = next_partner<2>(p, s_nb[w], s_lf[w], base, q1, i, j, k, q, e, nb, lc);
                    if (!__any_sync(0xffffffffu, kind != 0)) break;
                    if (kind != 0) rev2(entry_dx(e), entry_dy(e), entry_dz(e), kind == 2, (long long)nb * kCells + lc);
                    q++;
                }
            } else {
#pragma unroll 1
                for (int q = q0; q < q1; q++) {
                    const int e = __ldg(p.entries + base + q);
                    const int sx = i + entry_dx(e), sy = j + entry_dy(e), sz = k + entry_dz(e);
                    const int slot = ((sx >> 3) + 1) + 3 * ((sy >> 3) + 1) + 9 * ((sz >> 3) + 1);
                    const int nb = s_nb[w][slot];
                    if (nb < 0) continue;
                    const bool pleaf = s_lf[w][slot] != 0;
                    if (!pleaf && entry_near(e)) continue;
                    rev2(entry_dx(e), entry_dy(e), entry_dz(e), pleaf,
                         (long long)nb * kCells + (sx & 7) + 8 * (sy & 7) + 64 * (sz & 7));
                }
            }
        }
        // this cell's target-side adjoints (the correction's mass ratio, after
        // pass 2) and centre-of-mass adjoint (both passes)
        if (!cleaf) {
            if (passes & 2) {
                // the octupole's adjoint once per target, in the item that
                // starts its pass-2 range: dJ/dM3_A = -(1 / m_A) h^-3 al .
                // sum_B m_B D4(R'_B), al = -(G/6) h^-2 a, from the quartic sum
                // of all its pairs that the forward pass kept
                if (am && mC != 0.0 && q0 == 0) {
                    double aC[3];
#pragma unroll
                    for (int r = 0; r < 3; r++) aC[r] = sA * locbar[(20 + r) * N + cell];
#pragma unroll
                    for (int r = 0; r < 15; r++) acc.A4[r] = p.a4_out[r * N + cell];
                    reverse_target_finish(acc, aC, -hi3 / mC);
#pragma unroll
                    for (int r = 0; r < 10; r++) atomicAdd(mombar + (10 + r) * N + cell, acc.M3A[r]);
                }
                atomicAdd(mombar + cell, acc.mA);
            }
#pragma unroll
            for (int s = 0; s < 3; s++) atomicAdd(mombar + (1 + s) * N + cell, acc.R[s]);
        }
        __syncwarp();
    }
}

// M2M reverse at parent level: 8 lanes per parent cell, one per child (one
// warp = 4 parent cells, 128 blocks per node); each lane writes its child.  Forward (parent units, child offsets d = X_k - X_P):
//   M = sum m_k,  X_P = sum m_k X_k / M,  M2 = sum M2_k + m_k d d,
//   M3 = sum M3_k + 3 sym(M2_k d) + m_k d d d,
// so with the parent's adjoints (Bm, BX, B2, B3) each child gathers
//   M3bar_k += B3,  M2bar_k += B2 + 3 B3 d,  mbar_k += B2:dd + B3:ddd,
//   dbar = 2 m_k B2 d + 3 B3:M2_k + 3 m_k B3:dd,
// and then the centre of mass: Xbar_k += Xtot m_k / M, mbar_k += Xtot.d / M
// + Bm with Xtot = BX - sum dbar (the geometric centre, a constant, when
// M = 0), Xtot summed over the 8 lanes.
__global__ void __launch_bounds__(32) k_m2m_reverse(DevTree t, int first, double* mombar) {
    const int node = first + (blockIdx.x >> 7);
    const int child0 = t.node_child[node];
    if (child0 < 0) return;
    const long long N = t.n_cells;
    const int L = t.node_level[node];
    const double hp = t.size / (double)(8 << L), hc = 0.5 * hp;
    const int c = ((blockIdx.x & 127) << 2) + (threadIdx.x >> 3);  // parent cell in the node
    const int q = threadIdx.x & 7;                                  // child octant
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const long long pcell = (long long)node * kCells + c;
    const double M = t.mom64[pcell];
    const double XP[3] = {t.mom64[N + pcell], t.mom64[2 * N + pcell], t.mom64[3 * N + pcell]};
    const double Bm = mombar[pcell];
    double B2[6], B3[10];
#pragma unroll
    for (int r = 0; r < 6; r++) B2[r] = mombar[(4 + r) * N + pcell];
#pragma unroll
    for (int r = 0; r < 10; r++) B3[r] = mombar[(10 + r) * N + pcell];
    const int cn = child0 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2);
    const int a = q & 1, b = (q >> 1) & 1, e = q >> 2;
    const long long cc = (long long)cn * kCells + (2 * (i & 3) + a) + 8 * (2 * (j & 3) + b) +
                         64 * (2 * (k & 3) + e);
    const double d[3] = {hp * (0.5 * ((a - 0.5) + t.mom64[N + cc]) - XP[0]),
                         hp * (0.5 * ((b - 0.5) + t.mom64[2 * N + cc]) - XP[1]),
                         hp * (0.5 * ((e - 0.5) + t.mom64[3 * N + cc]) - XP[2])};
    const double m = t.mom64[cc];
    double M2k[6];
#pragma unroll
    for (int r = 0; r < 6; r++) M2k[r] = hc * hc * t.mom64[(4 + r) * N + cc];
    // M2bar_k += B2 + 3 B3 d
    double B3d[6];
    sym3_vec(B3, d, B3d);
    // mbar_k += B2 : dd + B3 : ddd
    double B2d[3], B3dd[3], B3M2[3];
    sym2_vec(B2, d, B2d);
    sym3_rr(B3, d, B3dd);
    sym3_contract(B3, M2k[0], M2k[3], M2k[5], 2.0 * M2k[1], 2.0 * M2k[2], 2.0 * M2k[4], B3M2);
    const double dd = B2d[0] * d[0] + B2d[1] * d[1] + B2d[2] * d[2];
    const double ddd = B3dd[0] * d[0] + B3dd[1] * d[1] + B3dd[2] * d[2];
    // dbar = 2 m B2 d + 3 B3 : M2_k + 3 m B3 : dd, and Xtot = BX - sum dbar
    double db[3], Xtot[3];
#pragma unroll
    for (int p = 0; p < 3; p++) db[p] = 2.0 * m * B2d[p] + 3.0 * B3M2[p] + 3.0 * m * B3dd[p];
#pragma unroll
    for (int p = 0; p < 3; p++) Xtot[p] = mombar[(1 + p) * N + pcell] - sum8(db[p]);  // every lane
    // the centre of mass X_P = sum m_k X_k / M and M = sum m_k
    const double iM = M != 0.0 ? 1.0 / M : 0.0;
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < 3; p++) {
        mombar[(1 + p) * N + cc] += db[p] + Xtot[p] * m * iM;
        s += Xtot[p] * d[p] * iM;
    }
    mombar[cc] += (dd + ddd) + (s + Bm);
#pragma unroll
    for (int n = 0; n < 6; n++) mombar[(4 + n) * N + cc] += B2[n] + 3.0 * B3d[n];
#pragma unroll
    for (int n = 0; n < 10; n++) mombar[(10 + n) * N + cc] += B3[n];
}

__global__ void __launch_bounds__(256) k_rho_bar(DevTree t, const int* __restrict__ leaf_node,
                                                 const double* __restrict__ mombar,
                                                 const double* __restrict__ w1, double* drho,
                                                 double G, int self_term) {
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    const int L = t.node_level[node];
    const double h = t.size / (double)(8 << L);
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
        const long long o = (long long)leaf * kCells + c;
        double v = mombar[(long long)node * kCells + c] * h * h * h;
        if (self_term) v += -G * h * h * cube_self_c() * w1[o];
        drho[o] = v;
    }
}

}  // namespace

void launch_adj_seed(const DevTree& t, const int* leaf_node, const double* w1, const double* w2,
                     double* locbar, cudaStream_t s) {
    k_adj_seed<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, w1, w2, locbar);
}

void launch_l2l_reverse(const DevTree& t, int first, int count, double* locbar, double* mombar,
                        cudaStream_t s) {
    if (count > 0) k_l2l_reverse<<<count * 128, 32, 0, s>>>(t, first, locbar, mombar);
}

void launch_m2l_reverse(const DevTree& t, const DevPlan& p, const double* locbar, double* mombar,
                        double G, int am, int ctas, cudaStream_t s) {
    k_m2l_reverse<<<ctas, 128, 0, s>>>(t, p, locbar, mombar, G, am);
}

void launch_m2m_reverse(const DevTree& t, int first, int count, double* mombar, cudaStream_t s) {
    if (count > 0) k_m2m_reverse<<<count * 128, 32, 0, s>>>(t, first, mombar);
}

void launch_rho_bar(const DevTree& t, const int* leaf_node, const double* mombar, const double* w1,
                    double* drho, double G, int self_term, cudaStream_t s) {
    k_rho_bar<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, mombar, w1, drho, G, self_term);
}

}  // namespace otfmm
