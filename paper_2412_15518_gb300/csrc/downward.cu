// Downward pass of the FMM gravity solve on GB300: L2L shifts and evaluation.
//
// Each cell's degree-3 local expansion (L0, L1, L2, L3 about its centre of
// mass) receives the exact shift of its parent's expansion by
// delta = X_cell - X_parent, and inherits the parent's angular-momentum
// correction acceleration (Sec. 4.3.1).  At a leaf cell (X = cell centre) the
// result is evaluated: phi = L0 (+ the optional uniform-cube self term) and
// g = -L1 + a_c.  One thread per cell, 8 blocks of 64 threads per node (so the
// coarse levels spread over many SMs), levels top-down, FP64 throughout.
#include "kernels.hpp"

namespace otfmm {

namespace {

// uniform cube of side 1 and density 1: int dV / |r| about its centre
// = 3 (ln(2 + sqrt 3) - pi / 6)
__host__ __device__ inline double cube_self_constant() {
    return 3.0 * (log(2.0 + sqrt(3.0)) - 3.14159265358979323846 / 6.0);
}

// 64 threads per block, 8 blocks per node (one z-layer of 64 cells each).
__global__ void __launch_bounds__(64) k_l2l(DevTree t, int first, const double* __restrict__ rho,
                                            double* __restrict__ phi, double* __restrict__ g,
                                            double G, int self_term) {
    const int node = first + (blockIdx.x >> 3);
    const int L = t.node_level[node];
    const int parent = t.node_parent[node];
    const int leaf = t.node_leaf[node];
    const long long N = t.n_cells;
    const double h = t.size / (double)(8 << L);
    const int* xyz = t.node_xyz + 3 * node;
    {
        const int c = ((blockIdx.x & 7) << 6) + threadIdx.x;
        const int ci[3] = {c & 7, (c >> 3) & 7, c >> 6};
        const long long cell = (long long)node * kCells + c;
        double E[kLoc];
        // a leaf cell's expansion holds only L0, L1 and the correction
#pragma unroll
        for (int r = 0; r < kLoc; r++)
            E[r] = (leaf < 0 || r < 4 || r >= 20) ? t.loc[r * N + cell] : 0.0;
        if (parent >= 0) {
            // parent cell and the cell's offset (0 or 1 per axis) inside it
            int pl = 0, off[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int gc = 8 * xyz[a] + ci[a];
                off[a] = gc & 1;
                pl += ((gc >> 1) & 7) << (3 * a);
            }
            const long long pcell = (long long)parent * kCells + pl;
            double P[kLoc];
#pragma unroll
            for (int r = 0; r < kLoc; r++) P[r] = t.loc[r * N + pcell];
            // delta = X_cell - X_parent in physical units (cell units of level L
            // times h): (off - 1/2) + dX_cell - 2 dX_parent
            double u[3];
#pragma unroll
            for (int a = 0; a < 3; a++)
                u[a] = h * ((off[a] - 0.5) + t.mom64[(1 + a) * N + cell] -
                            2.0 * t.mom64[(1 + a) * N + pcell]);
            const double x = u[0], y = u[1], z = u[2];
            const double* L2 = P + 4;
            const double* L3 = P + 10;
            // L2 . delta and L3 : delta delta
            const double A2x = fma(L2[0], x, fma(L2[1], y, L2[2] * z));
            const double A2y = fma(L2[1], x, fma(L2[3], y, L2[4] * z));
            const double A2z = fma(L2[2], x, fma(L2[4], y, L2[5] * z));
            const double xx = x * x, yy = y * y, zz = z * z, xy2 = 2 * x * y, xz2 = 2 * x * z,
                         yz2 = 2 * y * z;
            const double B3x = fma(L3[0], xx, fma(L3[3], yy, fma(L3[5], zz, fma(L3[1], xy2, fma(L3[2], xz2, L3[4] * yz2)))));
            const double B3y = fma(L3[1], xx, fma(L3[6], yy, fma(L3[8], zz, fma(L3[3], xy2, fma(L3[4], xz2, L3[7] * yz2)))));
            const double B3z = fma(L3[2], xx, fma(L3[7], yy, fma(L3[9], zz, fma(L3[4], xy2, fma(L3[5], xz2, L3[8] * yz2)))));
            // L0 += P0 + P1.d + d.P2.d / 2 + P3:ddd / 6
            E[0] += P[0] + fma(P[1], x, fma(P[2], y, P[3] * z)) +
                    0.5 * fma(A2x, x, fma(A2y, y, A2z * z)) +
                    (1.0 / 6.0) * fma(B3x, x, fma(B3y, y, B3z * z));
            // L1 += P1 + P2 d + P3:dd / 2
            E[1] += P[1] + A2x + 0.5 * B3x;
            E[2] += P[2] + A2y + 0.5 * B3y;
            E[3] += P[3] + A2z + 0.5 * B3z;
            if (leaf < 0) {
                // L2 += P2 + P3 . d ; L3 += P3
                E[4] += L2[0] + fma(L3[0], x, fma(L3[1], y, L3[2] * z));
                E[5] += L2[1] + fma(L3[1], x, fma(L3[3], y, L3[4] * z));
                E[6] += L2[2] + fma(L3[2], x, fma(L3[4], y, L3[5] * z));
                E[7] += L2[3] + fma(L3[3], x, fma(L3[6], y, L3[7] * z));
                E[8] += L2[4] + fma(L3[4], x, fma(L3[7], y, L3[8] * z));
                E[9] += L2[5] + fma(L3[5], x, fma(L3[8], y, L3[9] * z));
#pragma unroll
                for (int r = 0; r < 10; r++) E[10 + r] += L3[r];
            }
#pragma unroll
            for (int a = 0; a < 3; a++) E[20 + a] += P[20 + a];
        }
        if (leaf < 0) {
#pragma unroll
            for (int r = 0; r < kLoc; r++) t.loc[r * N + cell] = E[r];
        } else {
            const long long o = (long long)leaf * kCells + c;
            double p = E[0];
            if (self_term) p += -G * h * h * cube_self_constant() * rho[o];
            phi[o] = p;
#pragma unroll
            for (int a = 0; a < 3; a++) g[((long long)leaf * 3 + a) * kCells + c] = -E[1 + a] + E[20 + a];
        }
    }
}

}  // namespace

void launch_l2l(const DevTree& t, int level, int first, int count, const double* rho,
                double* phi, double* g, double G, int self_term, cudaStream_t s) {
    (void)level;
    if (count > 0) k_l2l<<<count * 8, 64, 0, s>>>(t, first, rho, phi, g, G, self_term);
}

}  // namespace otfmm
