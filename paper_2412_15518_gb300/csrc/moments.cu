// Upward pass of the FMM gravity solve on GB300: leaf masses and exact M2M.
//
// A leaf cell is a point mass m = rho h^3 at its centre (its offset dX,
// M2 and M3 are zero and are written once when the tree is built).  An
// interior cell's moments are the exact moments of its 8 children about the
// parent's centre of mass (multipole moments up to order 3, implied by the
// FMM of Sec. 4.3.2).  Everything is FP64; an FP32 copy is written for the
// FP32-bulk interaction form.  One thread per cell, one block per node, all
// loads and stores structure-of-arrays and coalesced across the block.
#include "kernels.hpp"

namespace otfmm {

namespace {

__global__ void __launch_bounds__(256) k_leaf_moments(DevTree t, const int* __restrict__ leaf_node,
                                                      const double* __restrict__ rho) {
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    const int L = t.node_level[node];
    const double h = t.size / (double)(8 << L);
    const double h3 = h * h * h;
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
        const double m = rho[(long long)leaf * kCells + c] * h3;
        const long long cell = (long long)node * kCells + c;
        t.mom64[cell] = m;
        t.mom32[cell] = (float)m;
    }
}

// (i, j, k) of the 10 packed components of a symmetric rank-3 tensor
__constant__ int c_t3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};

__device__ __forceinline__ int p2(int i, int j) {
    // packed index of (i, j) in xx xy xz yy yz zz
    return i <= j ? (i == 0 ? j : (i == 1 ? 2 + j : 5)) : (j == 0 ? i : (j == 1 ? 2 + i : 5));
}

__global__ void __launch_bounds__(256) k_m2m(DevTree t, int first) {
    const int node = first + blockIdx.x;
    const int child0 = t.node_child[node];
    if (child0 < 0) return;  // leaf node: moments come from rho
    const long long N = t.n_cells;
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
        const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
        // the 8 children of cell (i, j, k) lie in child node (i>>2, j>>2, k>>2)
        const int cn = child0 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2);
        const long long cbase = (long long)cn * kCells;
        double m[8], pos[8][3];
        double M = 0.0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int a = q & 1, b = (q >> 1) & 1, e = q >> 2;
            const long long cc = cbase + (2 * (i & 3) + a) + 8 * (2 * (j & 3) + b) + 64 * (2 * (k & 3) + e);
            m[q] = t.mom64[cc];
            // child centre of mass relative to the parent cell centre, parent units
            pos[q][0] = 0.5 * ((a - 0.5) + t.mom64[N + cc]);
            pos[q][1] = 0.5 * ((b - 0.5) + t.mom64[2 * N + cc]);
            pos[q][2] = 0.5 * ((e - 0.5) + t.mom64[3 * N + cc]);
            M += m[q];
        }
        double X[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int q = 0; q < 8; q++)
#pragma unroll
            for (int a = 0; a < 3; a++) X[a] = fma(m[q], pos[q][a], X[a]);
        const double iM = 1.0 / M;
#pragma unroll
        for (int a = 0; a < 3; a++) X[a] *= iM;
        double S2[6] = {0, 0, 0, 0, 0, 0}, S3[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int a = q & 1, b = (q >> 1) & 1, e = q >> 2;
            const long long cc = cbase + (2 * (i & 3) + a) + 8 * (2 * (j & 3) + b) + 64 * (2 * (k & 3) + e);
            const double d[3] = {pos[q][0] - X[0], pos[q][1] - X[1], pos[q][2] - X[2]};
            double c2[6];
#pragma unroll
            for (int r = 0; r < 6; r++) c2[r] = 0.25 * t.mom64[(4 + r) * N + cc];  // child units -> parent
#pragma unroll
            for (int r = 0; r < 6; r++) {
                const int ii = r < 3 ? 0 : (r < 5 ? 1 : 2);
                const int jj = r < 3 ? r : (r < 5 ? r - 2 : 2);
                S2[r] += c2[r] + m[q] * d[ii] * d[jj];
            }
#pragma unroll
            for (int r = 0; r < 10; r++) {
                const int ii = c_t3[r][0], jj = c_t3[r][1], kk = c_t3[r][2];
                S3[r] += 0.125 * t.mom64[(10 + r) * N + cc] + c2[p2(ii, jj)] * d[kk] +
                         c2[p2(ii, kk)] * d[jj] + c2[p2(jj, kk)] * d[ii] +
                         m[q] * d[ii] * d[jj] * d[kk];
            }
        }
        const long long cell = (long long)node * kCells + c;
        t.mom64[cell] = M;
        t.mom32[cell] = (float)M;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            t.mom64[(1 + a) * N + cell] = X[a];
            t.mom32[(1 + a) * N + cell] = (float)X[a];
        }
#pragma unroll
        for (int r = 0; r < 6; r++) {
            t.mom64[(4 + r) * N + cell] = S2[r];
            t.mom32[(4 + r) * N + cell] = (float)S2[r];
        }
#pragma unroll
        for (int r = 0; r < 10; r++) {
            t.mom64[(10 + r) * N + cell] = S3[r];
            t.mom32[(10 + r) * N + cell] = (float)S3[r];
        }
    }
}

}  // namespace

void launch_leaf_moments(const DevTree& t, const int* leaf_node, const double* rho,
                         cudaStream_t s) {
    k_leaf_moments<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, rho);
}

void launch_m2m(const DevTree& t, int level, int first, int count, cudaStream_t s) {
    (void)level;
    if (count > 0) k_m2m<<<count, 256, 0, s>>>(t, first);
}

}  // namespace otfmm
