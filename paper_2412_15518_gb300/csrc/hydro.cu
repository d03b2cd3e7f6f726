// Right-hand side of the hydro solver on a uniform grid of 8^3 sub-grids:
// dU/dt of the conserved fields U = (rho, s, E) of an ideal gas from the
// finite-volume fluxes through every cell face and the gravity source (Sec. 2:
// Octo-Tiger's finite-volume hydrodynamics with PPM values at all 26
// directions of a cell; Sec. 4.3.1: the hydro solver beside the gravity
// solve in every Runge-Kutta stage).
//
// The 26 directional values come from the PPM kernel (ppm.cu).  The flux
// through a face is the 2-D Simpson rule over the face: the point at offset
// (e_a + s1 t1 + s2 t2) / 2 from the left cell's centre sees the left cell's
// value in direction e_a + s1 t1 + s2 t2 and the right cell's value in
// direction -e_a + s1 t1 + s2 t2 (t1 = e_{a+1}, t2 = e_{a+2}), weights
// (1, 4, 1) x (1, 4, 1) / 36; at each point the local Lax-Friedrichs
// (Rusanov) flux F* = (F(U_L) + F(U_R)) / 2 - a (U_R - U_L) / 2 with a the
// larger of |v_a| + c of the two states, c = sqrt(max(gamma p / rho, 0)).  A
// face on the domain boundary takes the inside state on both sides.  Then
// dU/dt = sum_a (F_low - F_high) / h + (0, rho g, s.g).
//
// One CTA per leaf sub-grid: for each axis the fluxes of the sub-grid's
// 9 x 8 x 8 faces go to shared memory (a boundary face of the sub-grid reads
// the neighbouring leaf's values, so it is computed by both leaves), then
// each cell adds its low face minus its high face.  The arithmetic is written
// operation by operation with round-to-nearest intrinsics and no fused
// multiply-add, in a fixed order, so that it equals a plain FP64 statement of
// the same formulas.
#include <cuda_runtime.h>

#include "common.cuh"
#include "hydro.hpp"

namespace otfmm {
namespace {

constexpr int kNF = 5;            // rho, s_x, s_y, s_z, E
constexpr int kFaces = 9 * 8 * 8;  // faces of a sub-grid along one axis

__device__ __forceinline__ int dir_index(int ox, int oy, int oz) {
    const int s = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
    return s < 13 ? s : s - 1;
}

// Euler flux along axis A of the state U and its wave speed |v_A| + c.
template <int A>
__device__ __forceinline__ double state_flux(const double* U, double gamma, double gm1, double* F) {
    const double rinv = __drcp_rn(U[0]);
    const double vx = __dmul_rn(U[1], rinv), vy = __dmul_rn(U[2], rinv), vz = __dmul_rn(U[3], rinv);
    const double ke = __dmul_rn(0.5, __dadd_rn(__dadd_rn(__dmul_rn(U[1], vx), __dmul_rn(U[2], vy)),
                                               __dmul_rn(U[3], vz)));
    const double p = __dmul_rn(gm1, __dsub_rn(U[4], ke));
    const double c = __dsqrt_rn(fmax(__dmul_rn(__dmul_rn(gamma, p), rinv), 0.0));
    const double s = U[1 + A];
    const double v = A == 0 ? vx : (A == 1 ? vy : vz);
    F[0] = s;
    F[1] = __dmul_rn(s, vx);
    F[2] = __dmul_rn(s, vy);
    F[3] = __dmul_rn(s, vz);
    F[4] = __dmul_rn(__dadd_rn(U[4], p), v);
    F[1 + A] = __dadd_rn(F[1 + A], p);
    return __dadd_rn(fabs(v), c);
}

// The fluxes of the sub-grid's faces along axis A into sF[face][field]:
// face (fa, cell coordinates across A), left cell fa - 1 and right cell fa
// along A, each in its own leaf (s_lf: leaves of the 27 neighbour slots).
template <int A>
__device__ __forceinline__ void face_fluxes(const double* __restrict__ V, const int* s_lf, double gamma,
                                            double gm1, double* sF) {
    constexpr int T1 = (A + 1) % 3, T2 = (A + 2) % 3;
    for (int idx = threadIdx.x; idx < kFaces; idx += blockDim.x) {
        // cell index along x fastest, so that a warp's loads are consecutive
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
        const int cellL = c[0] + 8 * c[1] + 64 * c[2] + (fa == 0 ? 7 : fa - 1) * (A == 0 ? 1 : (A == 1 ? 8 : 64));
        const int cellR = c[0] + 8 * c[1] + 64 * c[2] + (fa == 8 ? 0 : fa) * (A == 0 ? 1 : (A == 1 ? 8 : 64));
        constexpr int kStep = A == 0 ? 1 : (A == 1 ? 3 : 9);  // neighbour slot step along A
        const int lfL = s_lf[13 - (fa == 0 ? kStep : 0)];
        const int lfR = s_lf[13 + (fa == 8 ? kStep : 0)];
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
            // a face on the domain boundary: the inside state on both sides
            const long long bL = lfL >= 0 ? ((long long)lfL * kNF * 26 + kL) * kCells + cellL
                                          : ((long long)lfR * kNF * 26 + kR) * kCells + cellR;
            const long long bR = lfR >= 0 ? ((long long)lfR * kNF * 26 + kR) * kCells + cellR : bL;
            double UL[kNF], UR[kNF];
#pragma unroll
            for (int f = 0; f < kNF; f++) {
                UL[f] = __ldg(V + bL + (long long)f * 26 * kCells);
                UR[f] = __ldg(V + bR + (long long)f * 26 * kCells);
            }
            double FL[kNF], FR[kNF];
            const double cl = state_flux<A>(UL, gamma, gm1, FL);
            const double cr = state_flux<A>(UR, gamma, gm1, FR);
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
#pragma unroll
        for (int f = 0; f < kNF; f++) sF[idx * kNF + f] = acc[f];
    }
}

// d += flux through the cell's low face - flux through its high face, axis A.
template <int A>
__device__ __forceinline__ void divergence(const double* sF, double (*d)[kNF]) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int cell = threadIdx.x + 256 * q;
        const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
        const int lo = A == 0 ? x + 9 * (y + 8 * z) : (A == 1 ? x + 8 * (y + 9 * z) : x + 8 * (y + 8 * z));
        const int hi = lo + (A == 0 ? 1 : (A == 1 ? 8 : 64));
#pragma unroll
        for (int f = 0; f < kNF; f++)
            d[q][f] = __dadd_rn(d[q][f], __dsub_rn(sF[lo * kNF + f], sF[hi * kNF + f]));
    }
}

__global__ void __launch_bounds__(256) k_hydro_rhs(DevTree t, const int* __restrict__ leaf_node,
                                                    const double* __restrict__ V,
                                                    const double* __restrict__ u,
                                                    const double* __restrict__ g, double gamma, double hinv,
                                                    double* __restrict__ out) {
    __shared__ double sF[kFaces * kNF];
    __shared__ int s_lf[27];
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    if (threadIdx.x < 27) {
        const int nb = t.nbr[(long long)node * 27 + threadIdx.x];
        s_lf[threadIdx.x] = nb >= 0 ? t.node_leaf[nb] : -1;
    }
    const double gm1 = __dsub_rn(gamma, 1.0);
    double d[2][kNF];
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
        for (int f = 0; f < kNF; f++) d[q][f] = 0.0;
    __syncthreads();
    face_fluxes<0>(V, s_lf, gamma, gm1, sF);
    __syncthreads();
    divergence<0>(sF, d);
    __syncthreads();  // the face buffer is rewritten for the next axis
    face_fluxes<1>(V, s_lf, gamma, gm1, sF);
    __syncthreads();
    divergence<1>(sF, d);
    __syncthreads();
    face_fluxes<2>(V, s_lf, gamma, gm1, sF);
    __syncthreads();
    divergence<2>(sF, d);
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int cell = threadIdx.x + 256 * q;
        double r[kNF];
#pragma unroll
        for (int f = 0; f < kNF; f++) r[f] = __dmul_rn(d[q][f], hinv);
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

}  // namespace

void launch_hydro_rhs(const DevTree& t, const int* leaf_node, const double* V, const double* u,
                      const double* g, double gamma, double h, double* dudt, cudaStream_t s) {
    if (t.n_leaf > 0)
        k_hydro_rhs<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, V, u, g, gamma, 1.0 / h, dudt);
}

}  // namespace otfmm
