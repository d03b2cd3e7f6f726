// PPM reconstruction of the hydro solver's 26 directional cell values (the
// second workload on the same octree of 8^3 sub-grids: Sec. 2, Octo-Tiger's
// finite-volume hydrodynamics computes the values at all 26 spatial
// directions of a grid cell with the piecewise parabolic method).
//
// For each of the 13 lines through a cell (the 26 neighbour offsets up to
// sign), 1-D PPM (Colella & Woodward 1984) on the cell averages along the
// line: the boundary value between neighbours i and i+1 is
// 7/12 (a_i + a_{i+1}) - 1/12 (a_{i-1} + a_{i+2}), held between a_i and
// a_{i+1}; then the parabola constraints -- both values set to the average at
// a local extremum, else the overshooting side replaced by 3a - 2(other) --
// give the cell's values toward -e and +e.  Cells outside the domain
// continue the averages by clamping each index into the grid.
//
// One CTA per leaf sub-grid: the sub-grid and 2 ghost layers (12^3 cells of
// one field) are staged in shared memory from the same-level neighbours;
// then, line by line, the boundary values between neighbouring cells are
// computed once each into shared memory (a cell's value toward +e is its
// neighbour's toward -e before limiting), and every cell limits its pair and
// writes its 2 of the 26 values, cell index fastest (coalesced).  The
// arithmetic is written operation by operation with round-to-nearest
// intrinsics and no fused multiply-add, in a fixed order, so that the
// limiter's comparisons see the same values as a plain FP64 statement.
#include <cuda_runtime.h>

#include "common.cuh"
#include "ppm.hpp"

namespace otfmm {
namespace {

constexpr int kG = 2;            // ghost layers
constexpr int kH = 8 + 2 * kG;   // halo side

__device__ __forceinline__ double interface_value(double am1, double a0, double a1, double a2) {
    const double v = __dsub_rn(__dmul_rn(7.0 / 12.0, __dadd_rn(a0, a1)), __dmul_rn(1.0 / 12.0, __dadd_rn(am1, a2)));
    return fmin(fmax(v, fmin(a0, a1)), fmax(a0, a1));
}

// Line e = (ex, ey, ez), first offset of the pair (e, -e): index kp for +e,
// km for -e (direction index of o = (ox+1) + 3 (oy+1) + 9 (oz+1), minus 1
// above 13).
struct Line {
    int ex, ey, ez, kp, km;
};
__device__ __forceinline__ int dir_index(int ox, int oy, int oz) {
    const int s = (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
    return s < 13 ? s : s - 1;
}

// Boundary-value box: positions p in [-1, 8] per axis (the cells' own
// boundaries p = c and their left ones p = c - e, for e of either sign),
// stored at p + 1.
constexpr int kI = 10;

__global__ void __launch_bounds__(256) k_ppm(DevTree t, const int* __restrict__ leaf_node,
                                              const double* __restrict__ u, int nf, int n_side,
                                              double* __restrict__ out) {
    __shared__ double halo[kH * kH * kH];
    __shared__ double bnd[2][kI * kI * kI];  // boundary values of two lines (double-buffered)
    __shared__ int s_lf[27];
    const int leaf = blockIdx.x;
    const int node = leaf_node[leaf];
    const int* xyz = t.node_xyz + 3 * node;
    if (threadIdx.x < 27) {
        const int nb = t.nbr[(long long)node * 27 + threadIdx.x];
        s_lf[threadIdx.x] = nb >= 0 ? t.node_leaf[nb] : -1;
    }
    // the 13 lines, each from its first offset in direction-index order
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
    for (int f = 0; f < nf; f++) {
        // stage the sub-grid and its ghosts (indices clamped into the domain)
        for (int h = threadIdx.x; h < kH * kH * kH; h += blockDim.x) {
            const int hx = h % kH, hy = (h / kH) % kH, hz = h / (kH * kH);
            int g[3] = {8 * xyz[0] + hx - kG, 8 * xyz[1] + hy - kG, 8 * xyz[2] + hz - kG};
            int slot = 0, cl = 0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                g[a] = g[a] < 0 ? 0 : (g[a] >= n_side ? n_side - 1 : g[a]);
                slot += ((g[a] >> 3) - xyz[a] + 1) * (a == 0 ? 1 : (a == 1 ? 3 : 9));
                cl += (g[a] & 7) << (3 * a);
            }
            const int lf = s_lf[slot];
            halo[h] = lf >= 0 ? u[((long long)lf * nf + f) * kCells + cl] : 0.0;
        }
        __syncthreads();
        double* o = out + ((long long)leaf * nf + f) * 26 * kCells;
#pragma unroll
        for (int l = 0; l < 13; l++) {
            const int ex = lines[l].ex, ey = lines[l].ey, ez = lines[l].ez;
            const int st = ex + kH * (ey + kH * ez);
            // boundary values between p and p + e for p in the box that the
            // cells' own (p = c) and left (p = c - e) boundaries cover
            const int lx = ex > 0 ? -1 : 0, ly = ey > 0 ? -1 : 0, lz = ez > 0 ? -1 : 0;
            const int nx = ex ? 9 : 8, ny = ey ? 9 : 8, nz = ez ? 9 : 8;
            double* I = bnd[l & 1];
            for (int q = threadIdx.x; q < nx * ny * nz; q += blockDim.x) {
                const int px = q % nx + lx, py = (q / nx) % ny + ly, pz = q / (nx * ny) + lz;
                const int h = (px + kG) + kH * ((py + kG) + kH * (pz + kG));
                I[(px + 1) + kI * ((py + 1) + kI * (pz + 1))] =
                    interface_value(halo[h - st], halo[h], halo[h + st], halo[h + 2 * st]);
            }
            __syncthreads();
            for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
                const int cx = c & 7, cy = (c >> 3) & 7, cz = c >> 6;
                const double a = halo[(cx + kG) + kH * ((cy + kG) + kH * (cz + kG))];
                double aR = I[(cx + 1) + kI * ((cy + 1) + kI * (cz + 1))];
                double aL = I[(cx - ex + 1) + kI * ((cy - ey + 1) + kI * (cz - ez + 1))];
                // parabola constraints
                const double ext = __dmul_rn(__dsub_rn(aR, a), __dsub_rn(a, aL));
                const double d = __dsub_rn(aR, aL);
                const double c6 = __dmul_rn(6.0, __dmul_rn(d, __dsub_rn(a, __dmul_rn(0.5, __dadd_rn(aL, aR)))));
                const double q6 = __dmul_rn(d, d);
                if (ext <= 0.0) {
                    aL = a;
                    aR = a;
                } else if (c6 > q6) {
                    aL = __dsub_rn(__dmul_rn(3.0, a), __dmul_rn(2.0, aR));
                } else if (-q6 > c6) {
                    aR = __dsub_rn(__dmul_rn(3.0, a), __dmul_rn(2.0, aL));
                }
                o[(long long)lines[l].kp * kCells + c] = aR;
                o[(long long)lines[l].km * kCells + c] = aL;
            }
            // the other buffer is written next; this one is rewritten two
            // lines on, after the next line's barrier
        }
        __syncthreads();  // the halo is restaged for the next field
    }
}

}  // namespace

void launch_ppm(const DevTree& t, const int* leaf_node, const double* u, int n_fields, int n_side,
                double* out, cudaStream_t s) {
    if (t.n_leaf > 0 && n_fields > 0) k_ppm<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, u, n_fields, n_side, out);
}

}  // namespace otfmm
