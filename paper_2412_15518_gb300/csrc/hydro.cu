// Right-hand side of the hydro solver on an octree of 8^3 sub-grids: dU/dt of
// the conserved fields U = (rho, s, E) of an ideal gas from the finite-volume
// fluxes through every cell face and the gravity source (Sec. 2: Octo-Tiger's
// finite-volume hydrodynamics with PPM values at all 26 directions of a cell;
// Sec. 4.3.1: mass, momentum and energy conserved across jumps in refinement level
// by matching the fluxes there; Sec. 4.3.1: the hydro solver beside the
// gravity solve in every Runge-Kutta stage).
//
// Three kernels, one CTA per leaf sub-grid each:
// * k_hydro_ppm: a halo of 3 ghost layers of every field at the leaf's level
//   (the same-level leaf's averages; across a refinement jump the mean of the
//   8 finer cells, or the average of the coarser cell that contains the ghost
//   cell; indices clamped into the domain), then PPM (Colella & Woodward
//   1984) along the 13 lines: the 26 values of the leaf's cells and the
//   values of the ghost cells next to its faces toward the leaf.
// * k_hydro_faces: the flux of every face of the leaf, the 2-D Simpson rule
//   over the face (weights (1, 4, 1) x (1, 4, 1) / 36) of the local
//   Lax-Friedrichs (Rusanov) flux F* = (F(U_L) + F(U_R)) / 2 - a (U_R - U_L) / 2,
//   a the larger of |v_a| + c of the two states, c = sqrt(max(gamma p / rho,
//   0)); a face on the domain boundary takes the inside state on both sides.
// * k_hydro_assemble: dU/dt = sum_a (F_low - F_high) / h_L + (0, rho g, s.g),
//   where a face of the leaf that borders a finer region takes the mean of
//   the 4 finer faces covering it (flux matching).
// The arithmetic is written operation by operation with round-to-nearest
// intrinsics and no fused multiply-add, in a fixed order, so that it equals
// a plain FP64 statement of the same formulas.
#include <cuda_runtime.h>

#include "common.cuh"
#include "hydro.hpp"

namespace otfmm {
namespace {

constexpr int kNF = 5;             // rho, s_x, s_y, s_z, E
constexpr int kFaces = 9 * 8 * 8;  // faces of a sub-grid along one axis
constexpr int kW = 3;              // ghost layers of the halo
constexpr int kHs = 8 + 2 * kW;    // halo side (local -3..10)
constexpr int kB = 12;             // boundary-value box side (positions -2..9)
constexpr int kGhost = 6 * 9 * 64; // ghost values per field: 6 sides x 9 directions x 64 cells

__device__ __forceinline__ int dir_index(int ox, int oy, int oz) {
    const int s = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
    return s < 13 ? s : s - 1;
}

__device__ __forceinline__ double interface_value(double am1, double a0, double a1, double a2) {
    const double v = __dsub_rn(__dmul_rn(7.0 / 12.0, __dadd_rn(a0, a1)), __dmul_rn(1.0 / 12.0, __dadd_rn(am1, a2)));
    return fmin(fmax(v, fmin(a0, a1)), fmax(a0, a1));
}

// Per-leaf lookup tables of the halo: for each of the 27 neighbour slots of
// the leaf's node, the same-level node's leaf (or -1), the leaves of its 8
// children when it is refined (or -1), and the leaf of the coarser node in
// the same slot of the parent's neighbourhood (or -1).
struct HaloTables {
    int lf[27];
    int kids[27][8];
    int plf[27];
    int refined[27];
};

__device__ void load_tables(const DevTree& t, int node, HaloTables& s) {
    const int parent = t.node_parent[node];
    for (int q = threadIdx.x; q < 27 * 8; q += blockDim.x) {
        const int slot = q >> 3, k = q & 7;
        const int nb = t.nbr[(long long)node * 27 + slot];
        const bool interior = nb >= 0 && t.node_leaf[nb] < 0;
        if (k == 0) {
            s.lf[slot] = nb >= 0 ? t.node_leaf[nb] : -1;
            s.refined[slot] = interior ? 1 : 0;
            const int pn = parent >= 0 ? t.nbr[(long long)parent * 27 + slot] : -1;
            s.plf[slot] = pn >= 0 ? t.node_leaf[pn] : -1;
        }
        s.kids[slot][k] = interior ? t.node_leaf[t.node_child[nb] + k] : -1;
    }
}

// Field f of the level-L cell at global index g (clamped into the domain) as
// seen from node xyz: the same-level leaf's average, the mean of the 8 finer
// cells (summed in z, y, x order), or the coarser cell's average.
__device__ double halo_value(const HaloTables& s, const double* __restrict__ u, const int* xyz,
                             const int* pxyz, int f, int gx, int gy, int gz, int* status) {
    const int slot = ((gx >> 3) - xyz[0] + 1) + 3 * ((gy >> 3) - xyz[1] + 1) + 9 * ((gz >> 3) - xyz[2] + 1);
    const int lf = s.lf[slot];
    if (lf >= 0) return __ldg(u + ((long long)lf * kNF + f) * kCells + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7));
    if (s.refined[slot]) {
        double sum = 0.0;
#pragma unroll
        for (int dz = 0; dz < 2; dz++)
#pragma unroll
            for (int dy = 0; dy < 2; dy++)
#pragma unroll
                for (int dx = 0; dx < 2; dx++) {
                    const int fx = 2 * gx + dx, fy = 2 * gy + dy, fz = 2 * gz + dz;
                    const int oct = ((fx >> 3) - 2 * (gx >> 3)) + 2 * ((fy >> 3) - 2 * (gy >> 3)) +
                                    4 * ((fz >> 3) - 2 * (gz >> 3));
                    const int kl = s.kids[slot][oct];
                    if (kl < 0) {  // not a 2:1-balanced tree: latched, no read
                        atomicOr(status, kStatusBadIndex);
                        continue;
                    }
                    sum = __dadd_rn(sum, __ldg(u + ((long long)kl * kNF + f) * kCells + (fx & 7) + 8 * (fy & 7) +
                                               64 * (fz & 7)));
                }
        return __dmul_rn(sum, 0.125);
    }
    // a coarser leaf: the cell at half the index, in the parent's neighbourhood
    const int cx = gx >> 1, cy = gy >> 1, cz = gz >> 1;
    const int pslot = ((cx >> 3) - pxyz[0] + 1) + 3 * ((cy >> 3) - pxyz[1] + 1) + 9 * ((cz >> 3) - pxyz[2] + 1);
    const int cl = pslot >= 0 && pslot < 27 ? s.plf[pslot] : -1;
    if (cl < 0) {
        atomicOr(status, kStatusBadIndex);
        return 0.0;
    }
    return __ldg(u + ((long long)cl * kNF + f) * kCells + (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7));
}

// Line e = (ex, ey, ez), its first offset's direction index kp and the
// opposite's km.
struct Line {
    int ex, ey, ez, kp, km;
};

// Halo and PPM values of one leaf: Vown [n_leaf][5][26][512] for its cells;
// Vgh [n_leaf][5][6][9][64] for the ghost cells next to its faces (side
// 2A + hi: local coordinate -1 or 8 along axis A; direction p = (s2 + 1) 3 +
// (s1 + 1) of o = (hi ? -1 : 1) e_A + s1 e_{A+1} + s2 e_{A+2}; cell q =
// c_{A+1} + 8 c_{A+2}).
__global__ void __launch_bounds__(256) k_hydro_ppm(DevTree t, const int* __restrict__ leaf_node,
                                                    const double* __restrict__ u, double* __restrict__ Vown,
                                                    double* __restrict__ Vgh) {
    __shared__ double halo[kHs * kHs * kHs];
    __shared__ double bnd[kB * kB * kB];
    __shared__ HaloTables s;
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    const int L = t.node_level[node];
    const int xyz[3] = {t.node_xyz[3 * node], t.node_xyz[3 * node + 1], t.node_xyz[3 * node + 2]};
    const int pxyz[3] = {xyz[0] >> 1, xyz[1] >> 1, xyz[2] >> 1};
    const int N = 8 << L;
    load_tables(t, node, s);
    Line lines[13];
    int nl = 0;
#pragma unroll
    for (int oz = -1; oz <= 1; oz++)
#pragma unroll
        for (int oy = -1; oy <= 1; oy++)
#pragma unroll
            for (int ox = -1; ox <= 1; ox++) {
                const int k = (ox || oy || oz) ? dir_index(ox, oy, oz) : -1;
                const int km = (ox || oy || oz) ? dir_index(-ox, -oy, -oz) : -1;
                if (k >= 0 && k < km) lines[nl++] = {ox, oy, oz, k, km};
            }
    __syncthreads();
    // The ghost cells next to a face need their own values only across a
    // refinement jump: across a same-level leaf they are that leaf's own
    // values (the same averages, the same arithmetic), which the faces kernel
    // reads there; across the domain boundary the face takes the inside state.
    bool need[6];
    const int top = (1 << L) - 1;
#pragma unroll
    for (int side = 0; side < 6; side++) {
        const int A = side >> 1, hi = side & 1;
        const int step = A == 0 ? 1 : (A == 1 ? 3 : 9);
        const bool boundary = hi ? xyz[A] == top : xyz[A] == 0;
        need[side] = !boundary && s.lf[13 + (hi ? step : -step)] < 0;
    }
    for (int f = 0; f < kNF; f++) {
        for (int h = threadIdx.x; h < kHs * kHs * kHs; h += blockDim.x) {
            const int hx = h % kHs, hy = (h / kHs) % kHs, hz = h / (kHs * kHs);
            int gx = 8 * xyz[0] + hx - kW, gy = 8 * xyz[1] + hy - kW, gz = 8 * xyz[2] + hz - kW;
            gx = gx < 0 ? 0 : (gx >= N ? N - 1 : gx);
            gy = gy < 0 ? 0 : (gy >= N ? N - 1 : gy);
            gz = gz < 0 ? 0 : (gz >= N ? N - 1 : gz);
            halo[h] = halo_value(s, u, xyz, pxyz, f, gx, gy, gz, t.status);
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < 13; l++) {
            const int ex = lines[l].ex, ey = lines[l].ey, ez = lines[l].ez;
            const int st = ex + kHs * (ey + kHs * ez);
            // boundary values between p and p + e for the positions p = c and
            // p = c - e of the leaf's cells and of the ghost cells it needs
            int lo[3], hi[3];
            {
                const int e[3] = {ex, ey, ez};
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    lo[a] = min(0, -e[a]);
                    hi[a] = max(7, 7 - e[a]);
                    if (need[2 * a]) lo[a] = min(lo[a], min(-1, -1 - e[a]));
                    if (need[2 * a + 1]) hi[a] = max(hi[a], max(8, 8 - e[a]));
                }
            }
            const int lx = lo[0], ly = lo[1], lz = lo[2];
            const int nx = hi[0] - lo[0] + 1, ny = hi[1] - lo[1] + 1, nz = hi[2] - lo[2] + 1;
            for (int q = threadIdx.x; q < nx * ny * nz; q += blockDim.x) {
                const int px = q % nx + lx, py = (q / nx) % ny + ly, pz = q / (nx * ny) + lz;
                const int h = (px + kW) + kHs * ((py + kW) + kHs * (pz + kW));
                bnd[(px + 2) + kB * ((py + 2) + kB * (pz + 2))] =
                    interface_value(halo[h - st], halo[h], halo[h + st], halo[h + 2 * st]);
            }
            __syncthreads();
            // the leaf's 512 cells, then the 6 x 64 ghost cells next to its faces
            for (int q = threadIdx.x; q < kCells + 384; q += blockDim.x) {
                int c[3];
                int side = -1, gq = 0;
                if (q < kCells) {
                    c[0] = q & 7;
                    c[1] = (q >> 3) & 7;
                    c[2] = q >> 6;
                } else {
                    side = (q - kCells) >> 6;
                    if (!need[side]) continue;
                    gq = (q - kCells) & 63;
                    const int A = side >> 1;
                    c[A] = (side & 1) ? 8 : -1;
                    c[A == 2 ? 0 : A + 1] = gq & 7;
                    c[A == 0 ? 2 : A - 1] = gq >> 3;
                    // a ghost cell keeps only a value toward the leaf: lines across the face
                    if ((A == 0 ? ex : (A == 1 ? ey : ez)) == 0) continue;
                }
                const double a = halo[(c[0] + kW) + kHs * ((c[1] + kW) + kHs * (c[2] + kW))];
                double aR = bnd[(c[0] + 2) + kB * ((c[1] + 2) + kB * (c[2] + 2))];
                double aL = bnd[(c[0] - ex + 2) + kB * ((c[1] - ey + 2) + kB * (c[2] - ez + 2))];
                // parabola constraints
                const double ext = __dmul_rn(__dsub_rn(aR, a), __dsub_rn(a, aL));
                const double dd = __dsub_rn(aR, aL);
                const double c6 = __dmul_rn(6.0, __dmul_rn(dd, __dsub_rn(a, __dmul_rn(0.5, __dadd_rn(aL, aR)))));
                const double q6 = __dmul_rn(dd, dd);
                if (ext <= 0.0) {
                    aL = a;
                    aR = a;
                } else if (c6 > q6) {
                    aL = __dsub_rn(__dmul_rn(3.0, a), __dmul_rn(2.0, aR));
                } else if (-q6 > c6) {
                    aR = __dsub_rn(__dmul_rn(3.0, a), __dmul_rn(2.0, aL));
                }
                if (side < 0) {
                    double* o = Vown + ((long long)leaf * kNF + f) * 26 * kCells;
                    o[(long long)lines[l].kp * kCells + q] = aR;
                    o[(long long)lines[l].km * kCells + q] = aL;
                } else {
                    // direction e carries aR, -e carries aL: the one pointing inward
                    const int A = side >> 1, inward = (side & 1) ? -1 : 1;
                    const int e[3] = {ex, ey, ez};
                    const int sg = e[A] == inward ? 1 : -1;
                    const int s1 = sg * e[A == 2 ? 0 : A + 1], s2 = sg * e[A == 0 ? 2 : A - 1];
                    const int p = (s2 + 1) * 3 + (s1 + 1);
                    Vgh[((((long long)leaf * kNF + f) * 6 + side) * 9 + p) * 64 + gq] = sg > 0 ? aR : aL;
                }
            }
            __syncthreads();  // bnd is rewritten by the next line, the halo by the next field
        }
    }
}

// The primitive variables of a state U: P = (v_x, v_y, v_z, p, c), c the
// sound speed, each operation correctly rounded (as the oracle evaluates it).
__device__ __forceinline__ void state_prims(const double* U, double gamma, double gm1, double* P) {
    const double rinv = __drcp_rn(U[0]);
    const double vx = __dmul_rn(U[1], rinv), vy = __dmul_rn(U[2], rinv), vz = __dmul_rn(U[3], rinv);
    const double ke = __dmul_rn(0.5, __dadd_rn(__dadd_rn(__dmul_rn(U[1], vx), __dmul_rn(U[2], vy)),
                                               __dmul_rn(U[3], vz)));
    const double p = __dmul_rn(gm1, __dsub_rn(U[4], ke));
    P[0] = vx;
    P[1] = vy;
    P[2] = vz;
    P[3] = p;
    P[4] = __dsqrt_rn(fmax(__dmul_rn(__dmul_rn(gamma, p), rinv), 0.0));
}

// Euler flux along axis A of the state U with primitives P, and its wave
// speed |v_A| + c.
template <int A>
__device__ __forceinline__ double prim_flux(const double* U, const double* P, double* F) {
    const double s = U[1 + A];
    const double v = P[A];
    F[0] = s;
    F[1] = __dmul_rn(s, P[0]);
    F[2] = __dmul_rn(s, P[1]);
    F[3] = __dmul_rn(s, P[2]);
    F[4] = __dmul_rn(__dadd_rn(U[4], P[3]), v);
    F[1 + A] = __dadd_rn(F[1 + A], P[3]);
    return __dadd_rn(fabs(v), P[4]);
}

// The primitives of every PPM value of the leaves' own cells, Vprim
// [n_leaf][5][26][512] beside Vown (component j of P for direction k of cell
// c at ((leaf 5 + j) 26 + k) 512 + c): each state's reciprocal and square root
// once, where the faces along the three axes use a corner value three times
// and an edge value twice.
__global__ void __launch_bounds__(256) k_hydro_prims(const double* __restrict__ Vown, double gamma,
                                                      double* __restrict__ Vprim) {
    const long long base = (long long)blockIdx.x * kNF * 26 * kCells;
    const double gm1 = __dsub_rn(gamma, 1.0);
    for (int idx = threadIdx.x; idx < 26 * kCells; idx += blockDim.x) {
        double U[kNF], P[kNF];
#pragma unroll
        for (int f = 0; f < kNF; f++) U[f] = __ldg(Vown + base + (long long)f * 26 * kCells + idx);
        state_prims(U, gamma, gm1, P);
#pragma unroll
        for (int f = 0; f < kNF; f++) Vprim[base + (long long)f * 26 * kCells + idx] = P[f];
    }
}

// Index of the face fa (0..8) along A of the cell coordinates c across A in
// a leaf's face list (cell index along x fastest).
template <int A>
__device__ __forceinline__ int face_index(int fa, const int* c) {
    return A == 0 ? fa + 9 * (c[1] + 8 * c[2]) : (A == 1 ? c[0] + 8 * (fa + 9 * c[2]) : c[0] + 8 * (c[1] + 8 * fa));
}

// The fluxes of the leaf's faces along axis A into F [n_leaf][3][576][5]:
// face fa between the cells fa - 1 and fa along A, the ghost cells' values
// at fa = 0 and 8; lo_bd / hi_bd: the leaf's low / high face along A lies on
// the domain boundary (the inside state on both sides).
template <int A>
__device__ __forceinline__ void leaf_faces(const double* __restrict__ Vown, const double* __restrict__ Vprim,
                                           const double* __restrict__ Vgh, int leaf, bool lo_bd, bool hi_bd,
                                           int lf_lo, int lf_hi, double gamma, double gm1,
                                           double* __restrict__ F, int* status) {
    constexpr int T1 = (A + 1) % 3, T2 = (A + 2) % 3;
    constexpr int kStA = A == 0 ? 1 : (A == 1 ? 8 : 64);
    for (int idx = threadIdx.x; idx < kFaces; idx += blockDim.x) {
        int c[3], fa;
        if (A == 0) {
            fa = idx % 9;
            c[1] = (idx / 9) & 7;
            c[2] = idx / 72;
        } else if (A == 1) {
            c[0] = idx & 7;
            fa = (idx >> 3) % 9;
            c[2] = idx / 72;
        } else {
            c[0] = idx & 7;
            c[1] = (idx >> 3) & 7;
            fa = idx >> 6;
        }
        c[A] = 0;
        const int base = c[0] + 8 * c[1] + 64 * c[2];
        // at the leaf's faces: the same-level neighbour's own cell (7 or 0
        // along A) where there is one, else the ghost cell's values
        const int cellL = base + (fa == 0 ? 7 : fa - 1) * kStA, cellR = base + (fa == 8 ? 0 : fa) * kStA;
        const int leafL = fa == 0 ? lf_lo : leaf, leafR = fa == 8 ? lf_hi : leaf;
        const bool ghL = fa == 0 && lf_lo < 0, ghR = fa == 8 && lf_hi < 0;
        const int gq = c[T1] + 8 * c[T2];
        double acc[kNF];
#pragma unroll
        for (int f = 0; f < kNF; f++) acc[f] = 0.0;
#pragma unroll 1
        for (int p = 0; p < 9; p++) {
            const int s1 = p % 3 - 1, s2 = p / 3 - 1;
            int o[3] = {0, 0, 0};
            o[T1] = s1;
            o[T2] = s2;
            o[A] = 1;
            const int kL = dir_index(o[0], o[1], o[2]);
            o[A] = -1;
            const int kR = dir_index(o[0], o[1], o[2]);
            // the states and their primitives: an own or same-level value's
            // from Vprim, a ghost value's formed here
            double UL[kNF], UR[kNF], PL[kNF], PR[kNF];
            const bool inL = !(fa == 0 && lo_bd), inR = !(fa == 8 && hi_bd);
#pragma unroll
            for (int f = 0; f < kNF; f++) {
                const long long lf = (long long)leaf * kNF + f;
                // (a ghost slot at the domain boundary is never read: the
                // inside state stands on both sides there)
                if (inL) {
                    if (ghL) {
                        UL[f] = __ldg(Vgh + ((lf * 6 + 2 * A) * 9 + p) * 64 + gq);
                    } else {
                        const long long o = (((long long)leafL * kNF + f) * 26 + kL) * kCells + cellL;
                        UL[f] = __ldg(Vown + o);
                        PL[f] = __ldg(Vprim + o);
                    }
                }
                if (inR) {
                    if (ghR) {
                        UR[f] = __ldg(Vgh + ((lf * 6 + 2 * A + 1) * 9 + p) * 64 + gq);
                    } else {
                        const long long o = (((long long)leafR * kNF + f) * 26 + kR) * kCells + cellR;
                        UR[f] = __ldg(Vown + o);
                        PR[f] = __ldg(Vprim + o);
                    }
                }
            }
            if (inL && ghL) state_prims(UL, gamma, gm1, PL);
            if (inR && ghR) state_prims(UR, gamma, gm1, PR);
            if (!inL)
#pragma unroll
                for (int f = 0; f < kNF; f++) {
                    UL[f] = UR[f];
                    PL[f] = PR[f];
                }
            if (!inR)
#pragma unroll
                for (int f = 0; f < kNF; f++) {
                    UR[f] = UL[f];
                    PR[f] = PL[f];
                }
            // a non-physical state is reported, not hidden (its rates are not finite)
            if (!(UL[0] > 0.0) || !(UR[0] > 0.0)) atomicOr(status, kStatusBadDensity);
            double FL[kNF], FR[kNF];
            const double cl = prim_flux<A>(UL, PL, FL);
            const double cr = prim_flux<A>(UR, PR, FR);
            const double half_a = __dmul_rn(0.5, fmax(cl, cr));
            // Simpson weights (1, 4, 1) x (1, 4, 1) / 36: centre, edges, corners
            const double w = p == 4 ? (4.0 * 4.0) / 36.0 : ((p & 1) ? (4.0 * 1.0) / 36.0 : (1.0 * 1.0) / 36.0);
#pragma unroll
            for (int f = 0; f < kNF; f++) {
                const double fs = __dsub_rn(__dmul_rn(0.5, __dadd_rn(FL[f], FR[f])),
                                            __dmul_rn(half_a, __dsub_rn(UR[f], UL[f])));
                acc[f] = __dadd_rn(acc[f], __dmul_rn(w, fs));
            }
        }
        double* o = F + (((long long)leaf * 3 + A) * kFaces + idx) * kNF;
#pragma unroll
        for (int f = 0; f < kNF; f++) o[f] = acc[f];
    }
}

__global__ void __launch_bounds__(256, 3) k_hydro_faces(DevTree t, const int* __restrict__ leaf_node,
                                                      const double* __restrict__ Vown,
                                                      const double* __restrict__ Vprim,
                                                      const double* __restrict__ Vgh, double gamma,
                                                      double* __restrict__ F) {
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    const int top = (1 << t.node_level[node]) - 1;
    const int* xyz = t.node_xyz + 3 * node;
    const double gm1 = __dsub_rn(gamma, 1.0);
    // the same-level leaf across each face (-1: none)
    int lf[6];
#pragma unroll
    for (int side = 0; side < 6; side++) {
        const int step = (side >> 1) == 0 ? 1 : ((side >> 1) == 1 ? 3 : 9);
        const int nb = t.nbr[(long long)node * 27 + 13 + ((side & 1) ? step : -step)];
        lf[side] = nb >= 0 ? t.node_leaf[nb] : -1;
    }
    leaf_faces<0>(Vown, Vprim, Vgh, leaf, xyz[0] == 0, xyz[0] == top, lf[0], lf[1], gamma, gm1, F,
                    t.status);
    leaf_faces<1>(Vown, Vprim, Vgh, leaf, xyz[1] == 0, xyz[1] == top, lf[2], lf[3], gamma, gm1, F,
                    t.status);
    leaf_faces<2>(Vown, Vprim, Vgh, leaf, xyz[2] == 0, xyz[2] == top, lf[4], lf[5], gamma, gm1, F,
                    t.status);
}

// d += F_low - F_high along A for the cell c of the leaf; a boundary face
// next to a finer region (ref[2A + hi]) takes the mean of the 4 finer faces
// that cover it, from the finer leaves' fluxes (fine[2A + hi][octant]).
template <int A>
__device__ __forceinline__ void add_axis(const double* __restrict__ F, int leaf, const int* c,
                                         const int (*fine)[8], const int* ref, int* status, double* d) {
    constexpr int T1 = (A + 1) % 3, T2 = (A + 2) % 3;
    double Fs[2][kNF];
#pragma unroll
    for (int hi = 0; hi < 2; hi++) {
        const int fa = c[A] + hi;
        if ((hi ? c[A] == 7 : c[A] == 0) && ref[2 * A + hi]) {
            // the finer cells next to the face: octant bit A toward this leaf
            double s[kNF];
#pragma unroll
            for (int f = 0; f < kNF; f++) s[f] = 0.0;
#pragma unroll
            for (int d2 = 0; d2 < 2; d2++)
#pragma unroll
                for (int d1 = 0; d1 < 2; d1++) {
                    const int f1 = 2 * c[T1] + d1, f2 = 2 * c[T2] + d2;
                    int fc[3];
                    fc[A] = 0;
                    fc[T1] = f1 & 7;
                    fc[T2] = f2 & 7;
                    int oct = (hi ? 0 : 1) << A;
                    oct |= (f1 >> 3) << T1;
                    oct |= (f2 >> 3) << T2;
                    const int fl = fine[2 * A + hi][oct];
                    if (fl < 0) {  // not a 2:1-balanced tree: latched, no read
                        atomicOr(status, kStatusBadIndex);
                        continue;
                    }
                    const double* p =
                        F + (((long long)fl * 3 + A) * kFaces + face_index<A>(hi ? 0 : 8, fc)) * kNF;
#pragma unroll
                    for (int f = 0; f < kNF; f++) s[f] = __dadd_rn(s[f], __ldg(p + f));
                }
#pragma unroll
            for (int f = 0; f < kNF; f++) Fs[hi][f] = __dmul_rn(s[f], 0.25);
        } else {
            const double* p = F + (((long long)leaf * 3 + A) * kFaces + face_index<A>(fa, c)) * kNF;
#pragma unroll
            for (int f = 0; f < kNF; f++) Fs[hi][f] = __ldg(p + f);
        }
    }
#pragma unroll
    for (int f = 0; f < kNF; f++) d[f] = __dadd_rn(d[f], __dsub_rn(Fs[0][f], Fs[1][f]));
}

// 1/h_L per level, computed on the host as 1 / (size / (8 2^L)).
struct HydroLevels {
    double hinv[kMaxLevels];
};

__global__ void __launch_bounds__(256) k_hydro_assemble(DevTree t, const int* __restrict__ leaf_node,
                                                         const double* __restrict__ F,
                                                         const double* __restrict__ u,
                                                         const double* __restrict__ g, HydroLevels lv,
                                                         double* __restrict__ out) {
    __shared__ int fine[6][8];
    __shared__ int ref[6];
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    if (threadIdx.x < 48) {
        const int side = threadIdx.x >> 3, k = threadIdx.x & 7, A = side >> 1;
        const int step = A == 0 ? 1 : (A == 1 ? 3 : 9);
        const int nb = t.nbr[(long long)node * 27 + 13 + ((side & 1) ? step : -step)];
        const bool interior = nb >= 0 && t.node_leaf[nb] < 0;
        fine[side][k] = interior ? t.node_leaf[t.node_child[nb] + k] : -1;
        if (k == 0) ref[side] = interior ? 1 : 0;
    }
    __syncthreads();
    const double hinv = lv.hinv[t.node_level[node]];
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int cell = threadIdx.x + 256 * q;
        const int c[3] = {cell & 7, (cell >> 3) & 7, cell >> 6};
        double d[kNF];
#pragma unroll
        for (int f = 0; f < kNF; f++) d[f] = 0.0;
        add_axis<0>(F, leaf, c, fine, ref, t.status, d);
        add_axis<1>(F, leaf, c, fine, ref, t.status, d);
        add_axis<2>(F, leaf, c, fine, ref, t.status, d);
        double r[kNF];
#pragma unroll
        for (int f = 0; f < kNF; f++) r[f] = __dmul_rn(d[f], hinv);
        if (g) {
            const long long cu = (long long)leaf * kNF * kCells + cell;
            const long long cg = (long long)leaf * 3 * kCells + cell;
            const double rho = u[cu], sx = u[cu + kCells], sy = u[cu + 2 * kCells], sz = u[cu + 3 * kCells];
            const double gx = g[cg], gy = g[cg + kCells], gz = g[cg + 2 * kCells];
            r[1] = __dadd_rn(r[1], __dmul_rn(rho, gx));
            r[2] = __dadd_rn(r[2], __dmul_rn(rho, gy));
            r[3] = __dadd_rn(r[3], __dmul_rn(rho, gz));
            r[4] = __dadd_rn(r[4], __dadd_rn(__dadd_rn(__dmul_rn(sx, gx), __dmul_rn(sy, gy)), __dmul_rn(sz, gz)));
        }
#pragma unroll
        for (int f = 0; f < kNF; f++) out[((long long)leaf * kNF + f) * kCells + cell] = r[f];
    }
}
// The density of the stage's state, rho[leaf][c] = U[leaf][0][c], for its
// gravity solve.
__global__ void k_stage_density(const double* __restrict__ U, double* __restrict__ rho, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rho[i] = U[(i / kCells) * kNF * kCells + (i % kCells)];
}

// One combination of the third-order strong-stability-preserving Runge-Kutta
// scheme (Shu & Osher 1988), in the order written: stage 1
// out = U0 + dt L; stage 2 out = 3/4 U0 + 1/4 (Uc + dt L); stage 3
// out = 1/3 U0 + 2/3 (Uc + dt L).
__global__ void k_rk3_combine(const double* __restrict__ U0, const double* Uc, const double* __restrict__ L,
                              double dt, int stage, double* out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dl = __dmul_rn(dt, L[i]);
    double v;
    if (stage == 1) v = __dadd_rn(U0[i], dl);
    else if (stage == 2) v = __dadd_rn(__dmul_rn(0.75, U0[i]), __dmul_rn(0.25, __dadd_rn(Uc[i], dl)));
    else v = __dadd_rn(__dmul_rn(1.0 / 3.0, U0[i]), __dmul_rn(2.0 / 3.0, __dadd_rn(Uc[i], dl)));
    out[i] = v;
}

}  // namespace

void launch_stage_density(const double* U, double* rho, int n_leaf, cudaStream_t s) {
    const long long n = (long long)n_leaf * kCells;
    if (n > 0) k_stage_density<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(U, rho, n);
}

void launch_rk3_combine(const double* U0, const double* Uc, const double* L, double dt, int stage, double* out,
                        int n_leaf, cudaStream_t s) {
    const long long n = (long long)n_leaf * kNF * kCells;
    if (n > 0) k_rk3_combine<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(U0, Uc, L, dt, stage, out, n);
}

size_t hydro_workspace_doubles(int n_leaf, size_t* own, size_t* ghost, size_t* faces) {
    *own = 2 * (size_t)n_leaf * kNF * 26 * kCells;  // the PPM values, then their primitives
    *ghost = (size_t)n_leaf * kNF * kGhost;
    *faces = (size_t)n_leaf * 3 * kFaces * kNF;
    return *own + *ghost + *faces;
}

void launch_hydro_rhs(const DevTree& t, const int* leaf_node, const double* u, const double* g, double gamma,
                      double* work, double* dudt, cudaStream_t s) {
    if (t.n_leaf <= 0) return;
    size_t own, ghost, faces;
    hydro_workspace_doubles(t.n_leaf, &own, &ghost, &faces);
    double* Vown = work;
    double* Vprim = work + own / 2;
    double* Vgh = work + own;
    double* F = Vgh + ghost;
    HydroLevels lv;
    for (int L = 0; L < kMaxLevels; L++) lv.hinv[L] = 1.0 / (t.size / (double)(8 << L));
    k_hydro_ppm<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, u, Vown, Vgh);
    k_hydro_prims<<<t.n_leaf, 256, 0, s>>>(Vown, gamma, Vprim);
    k_hydro_faces<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, Vown, Vprim, Vgh, gamma, F);
    k_hydro_assemble<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, F, u, g, lv, dudt);
}

}  // namespace otfmm
