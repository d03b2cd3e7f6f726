// Downward pass of the FMM gravity solve on GB300: L2L shifts and evaluation.
//
// Each cell's degree-3 local expansion (L0, L1, L2, L3 about its centre of
// mass) receives the exact shift of its parent's expansion by
// delta = X_cell - X_parent, and inherits the parent's angular-momentum
// correction acceleration (Sec. 4.3.1).  At a leaf cell (X = cell centre) the
// result is evaluated: phi = L0 (+ the optional uniform-cube self term) and
// g = -L1 + a_c.  One thread per cell, one warp per block (so the coarse
// levels spread over many SMs), levels top-down, FP64 throughout.
#include "kernels.hpp"

namespace otfmm {

namespace {

// uniform cube of side 1 and density 1: int dV / |r| about its centre
// = 3 (ln(2 + sqrt 3) - pi / 6)
__host__ __device__ inline double cube_self_constant() {
    return 3.0 * (log(2.0 + sqrt(3.0)) - 3.14159265358979323846 / 6.0);
}

// Adds the parent's expansion P shifted by delta = (x, y, z) to the
// expansion E of an interior cell (exact degree-3 shift, FP64):
//   L0 += P0 + P1.d + d.P2.d / 2 + P3:ddd / 6,  L1 += P1 + P2 d + P3:dd / 2,
//   L2 += P2 + P3 . d,  L3 += P3,  a_c += a_c(parent).
__device__ __forceinline__ void add_shift(double* E, const double* P, double x, double y, double z) {
    const double* L2 = P + 4;
    const double* L3 = P + 10;
    // L2 . delta and L3 : delta delta
    const double A2x = fma(L2[0], x, fma(L2[1], y, L2[2] * z));
    const double A2y = fma(L2[1], x, fma(L2[3], y, L2[4] * z));
    const double A2z = fma(L2[2], x, fma(L2[4], y, L2[5] * z));
    const double xx = x * x, yy = y * y, zz = z * z, xy2 = 2 * x * y, xz2 = 2 * x * z, yz2 = 2 * y * z;
    const double B3x = fma(L3[0], xx, fma(L3[3], yy, fma(L3[5], zz, fma(L3[1], xy2, fma(L3[2], xz2, L3[4] * yz2)))));
    const double B3y = fma(L3[1], xx, fma(L3[6], yy, fma(L3[8], zz, fma(L3[3], xy2, fma(L3[4], xz2, L3[7] * yz2)))));
    const double B3z = fma(L3[2], xx, fma(L3[7], yy, fma(L3[9], zz, fma(L3[4], xy2, fma(L3[5], xz2, L3[8] * yz2)))));
    E[0] += P[0] + fma(P[1], x, fma(P[2], y, P[3] * z)) + 0.5 * fma(A2x, x, fma(A2y, y, A2z * z)) +
            (1.0 / 6.0) * fma(B3x, x, fma(B3y, y, B3z * z));
    E[1] += P[1] + A2x + 0.5 * B3x;
    E[2] += P[2] + A2y + 0.5 * B3y;
    E[3] += P[3] + A2z + 0.5 * B3z;
    E[4] += L2[0] + fma(L3[0], x, fma(L3[1], y, L3[2] * z));
    E[5] += L2[1] + fma(L3[1], x, fma(L3[3], y, L3[4] * z));
    E[6] += L2[2] + fma(L3[2], x, fma(L3[4], y, L3[5] * z));
    E[7] += L2[3] + fma(L3[3], x, fma(L3[6], y, L3[7] * z));
    E[8] += L2[4] + fma(L3[4], x, fma(L3[7], y, L3[8] * z));
    E[9] += L2[5] + fma(L3[5], x, fma(L3[8], y, L3[9] * z));
#pragma unroll
    for (int r = 0; r < 10; r++) E[10 + r] += L3[r];
#pragma unroll
    for (int a = 0; a < 3; a++) E[20 + a] += P[20 + a];
}

// FP32-bulk form of add_shift: the shift's terms in delta (products of the
// parent's coefficients with delta) in FP32, every sum in FP64 -- the
// parent's coefficients are added exactly and each FP32 correction is
// widened exactly once.  The corrections are O(h / R) of the values they are
// added to, so their FP32 rounding stays far below the form's error.
__device__ __forceinline__ void add_shift_bulk(double* E, const double* P, float x, float y, float z) {
    float Q[20];
#pragma unroll
    for (int r = 1; r < 20; r++) Q[r] = (float)P[r];
    const float* L2 = Q + 4;
    const float* L3 = Q + 10;
    const float A2x = fmaf(L2[0], x, fmaf(L2[1], y, L2[2] * z));
    const float A2y = fmaf(L2[1], x, fmaf(L2[3], y, L2[4] * z));
    const float A2z = fmaf(L2[2], x, fmaf(L2[4], y, L2[5] * z));
    const float xx = x * x, yy = y * y, zz = z * z, xy2 = 2.f * x * y, xz2 = 2.f * x * z, yz2 = 2.f * y * z;
    const float B3x = fmaf(L3[0], xx, fmaf(L3[3], yy, fmaf(L3[5], zz, fmaf(L3[1], xy2, fmaf(L3[2], xz2, L3[4] * yz2)))));
    const float B3y = fmaf(L3[1], xx, fmaf(L3[6], yy, fmaf(L3[8], zz, fmaf(L3[3], xy2, fmaf(L3[4], xz2, L3[7] * yz2)))));
    const float B3z = fmaf(L3[2], xx, fmaf(L3[7], yy, fmaf(L3[9], zz, fmaf(L3[4], xy2, fmaf(L3[5], xz2, L3[8] * yz2)))));
    E[0] += P[0] + widen(fmaf(Q[1], x, fmaf(Q[2], y, Q[3] * z)) + 0.5f * fmaf(A2x, x, fmaf(A2y, y, A2z * z)) +
                         (1.0f / 6.0f) * fmaf(B3x, x, fmaf(B3y, y, B3z * z)));
    E[1] += P[1] + widen(fmaf(0.5f, B3x, A2x));
    E[2] += P[2] + widen(fmaf(0.5f, B3y, A2y));
    E[3] += P[3] + widen(fmaf(0.5f, B3z, A2z));
    E[4] += P[4] + widen(fmaf(L3[0], x, fmaf(L3[1], y, L3[2] * z)));
    E[5] += P[5] + widen(fmaf(L3[1], x, fmaf(L3[3], y, L3[4] * z)));
    E[6] += P[6] + widen(fmaf(L3[2], x, fmaf(L3[4], y, L3[5] * z)));
    E[7] += P[7] + widen(fmaf(L3[3], x, fmaf(L3[6], y, L3[7] * z)));
    E[8] += P[8] + widen(fmaf(L3[4], x, fmaf(L3[7], y, L3[8] * z)));
    E[9] += P[9] + widen(fmaf(L3[5], x, fmaf(L3[8], y, L3[9] * z)));
#pragma unroll
    for (int r = 0; r < 10; r++) E[10 + r] += P[10 + r];
#pragma unroll
    for (int a = 0; a < 3; a++) E[20 + a] += P[20 + a];
}

// 32 threads per block, 16 blocks per node.  The root is launched only when
// it is a leaf (an interior root has no parent expansion to add).  BULK: the
// FP32-bulk form's shift (add_shift_bulk).
template <bool BULK>
__global__ void __launch_bounds__(32) k_l2l(DevTree t, int first, const double* __restrict__ rho,
                                            double* __restrict__ phi, double* __restrict__ g,
                                            double G, int self_term) {
    const int node = first + (blockIdx.x >> 4);
    const int L = t.node_level[node];
    const int parent = t.node_parent[node];
    const int leaf = t.node_leaf[node];
    const long long N = t.n_cells;
    const double h = t.size / (double)(8 << L);
    const int* xyz = t.node_xyz + 3 * node;
    if (leaf >= 0 && parent >= 0) return;  // leaf cells of level >= 1: k_l2l_leafkids
    const int c = ((blockIdx.x & 15) << 5) + threadIdx.x;
    const int ci[3] = {c & 7, (c >> 3) & 7, c >> 6};
    const long long cell = (long long)node * kCells + c;
    double E[kLoc];
    // a leaf cell's expansion holds only L0, L1 and the correction
#pragma unroll
    for (int r = 0; r < kLoc; r++) E[r] = (leaf < 0 || r < 4 || r >= 20) ? t.loc[r * N + cell] : 0.0;
    if (parent >= 0) {  // an interior cell below the root
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
        if (BULK) {
            const float hf = (float)h;
            const float* mc = t.mom32 + cell * kMom;
            const float* mp = t.mom32 + pcell * kMom;
            float u[3];
#pragma unroll
            for (int a = 0; a < 3; a++) u[a] = hf * (((float)off[a] - 0.5f) + mc[1 + a] - 2.0f * mp[1 + a]);
            add_shift_bulk(E, P, u[0], u[1], u[2]);
        } else {
            double u[3];
#pragma unroll
            for (int a = 0; a < 3; a++)
                u[a] = h * ((off[a] - 0.5) + t.mom64[(1 + a) * N + cell] - 2.0 * t.mom64[(1 + a) * N + pcell]);
            add_shift(E, P, u[0], u[1], u[2]);
        }
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

// Packed index of (i, j, k) in a symmetric rank-3 tensor.
__device__ __forceinline__ int pk3(int i, int j, int k) {
    if (i > j) { const int s = i; i = j; j = s; }
    if (j > k) { const int s = j; j = k; k = s; }
    if (i > j) { const int s = i; i = j; j = s; }
    return i == 0 ? (j == 0 ? k : (j == 1 ? 2 + k : 5)) : (i == 1 ? (j == 1 ? 5 + k : 8) : 9);
}

// Values at the 8 corners s in {-1, 1}^3 (index bits x = 1, y = 2, z = 4, bit
// set means s = +1) of v(s) = sum_q c_q prod_{axes in q} s_axis, in place.
template <class T> __device__ __forceinline__ void corners8(T* c) {
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (!(q & bit)) {
                const double u = c[q], v = c[q | bit];
                c[q] = u - v;
                c[q | bit] = u + v;
            }
}

// Downward pass into leaf children: one thread per parent cell whose 8
// children are leaf cells.  The parent's expansion is shifted once to the
// parent cell centre (coefficients A); the children sit at e = eps s with
// eps = h/4 and s in {-1, 1}^3, so the degree-3 polynomial and its gradient
// at the 8 children are sums of a few coefficients with sign patterns:
//   phi(s) = A0 + eps A1.s + eps^2 s.A2.s / 2 + eps^3 A3:sss / 6
//   grad(s) = A1 + eps A2 s + eps^2 A3:ss / 2
// evaluated as 8-point sign transforms.  Each child adds its own-level
// terms (L0, L1, a_c) and the parent's correction acceleration (folded into
// the constant coefficient of the gradient).  8 blocks of 64 threads per node.
__global__ void __launch_bounds__(64) k_l2l_leafkids(DevTree t, int first,
                                                      const double* __restrict__ rho,
                                                      double* __restrict__ phi,
                                                      double* __restrict__ g, double G,
                                                      int self_term) {
    const int node = first + (blockIdx.x >> 3);
    const int child0 = t.node_child[node];
    if (child0 < 0) return;
    const long long N = t.n_cells;
    const int c = ((blockIdx.x & 7) << 6) + threadIdx.x;
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int cn = child0 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2);
    const int leaf = t.node_leaf[cn];
    if (leaf < 0) return;  // interior children: k_l2l at the next level
    const int L = t.node_level[node];
    const double h = t.size / (double)(8 << L);
    const long long pcell = (long long)node * kCells + c;
    double P[kLoc];
#pragma unroll
    for (int r = 0; r < kLoc; r++) P[r] = t.loc[r * N + pcell];
    // shift from the parent's centre of mass to its cell centre
    const double x = -h * t.mom64[N + pcell], y = -h * t.mom64[2 * N + pcell],
                 z = -h * t.mom64[3 * N + pcell];
    const double* L2 = P + 4;
    const double* L3 = P + 10;
    const double A2x = fma(L2[0], x, fma(L2[1], y, L2[2] * z));
    const double A2y = fma(L2[1], x, fma(L2[3], y, L2[4] * z));
    const double A2z = fma(L2[2], x, fma(L2[4], y, L2[5] * z));
    const double xx = x * x, yy = y * y, zz = z * z, xy2 = 2 * x * y, xz2 = 2 * x * z, yz2 = 2 * y * z;
    const double B3x = fma(L3[0], xx, fma(L3[3], yy, fma(L3[5], zz, fma(L3[1], xy2, fma(L3[2], xz2, L3[4] * yz2)))));
    const double B3y = fma(L3[1], xx, fma(L3[6], yy, fma(L3[8], zz, fma(L3[3], xy2, fma(L3[4], xz2, L3[7] * yz2)))));
    const double B3z = fma(L3[2], xx, fma(L3[7], yy, fma(L3[9], zz, fma(L3[4], xy2, fma(L3[5], xz2, L3[8] * yz2)))));
    double A[20];
    A[0] = P[0] + fma(P[1], x, fma(P[2], y, P[3] * z)) + 0.5 * fma(A2x, x, fma(A2y, y, A2z * z)) +
           (1.0 / 6.0) * fma(B3x, x, fma(B3y, y, B3z * z));
    A[1] = P[1] + A2x + 0.5 * B3x;
    A[2] = P[2] + A2y + 0.5 * B3y;
    A[3] = P[3] + A2z + 0.5 * B3z;
    A[4] = L2[0] + fma(L3[0], x, fma(L3[1], y, L3[2] * z));
    A[5] = L2[1] + fma(L3[1], x, fma(L3[3], y, L3[4] * z));
    A[6] = L2[2] + fma(L3[2], x, fma(L3[4], y, L3[5] * z));
    A[7] = L2[3] + fma(L3[3], x, fma(L3[6], y, L3[7] * z));
    A[8] = L2[4] + fma(L3[4], x, fma(L3[7], y, L3[8] * z));
    A[9] = L2[5] + fma(L3[5], x, fma(L3[8], y, L3[9] * z));
#pragma unroll
    for (int r = 0; r < 10; r++) A[10 + r] = L3[r];
    const double* A2 = A + 4;
    const double* A3 = A + 10;
    const double e1 = 0.25 * h, e2 = e1 * e1, e3 = e2 * e1;
    // potential: sign-pattern coefficients, then the 8 corner values
    double cp[8];
    cp[0] = A[0] + 0.5 * e2 * (A2[0] + A2[3] + A2[5]);
    cp[1] = e1 * A[1] + (e3 / 6.0) * (A3[0] + 3.0 * (A3[3] + A3[5]));
    cp[2] = e1 * A[2] + (e3 / 6.0) * (A3[6] + 3.0 * (A3[1] + A3[8]));
    cp[4] = e1 * A[3] + (e3 / 6.0) * (A3[9] + 3.0 * (A3[2] + A3[7]));
    cp[3] = e2 * A2[1];
    cp[5] = e2 * A2[2];
    cp[6] = e2 * A2[4];
    cp[7] = e3 * A3[4];
    corners8(cp);
    // gradient, one component at a time
    double cg[3][8];
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const int pa = p == 0 ? 0 : (p == 1 ? 1 : 2);  // packed (p, x)
        const int pb = p == 0 ? 1 : (p == 1 ? 3 : 4);  // packed (p, y)
        const int pc = p == 0 ? 2 : (p == 1 ? 4 : 5);  // packed (p, z)
        double* v = cg[p];
        v[0] = A[1 + p] + 0.5 * e2 * (A3[pk3(p, 0, 0)] + A3[pk3(p, 1, 1)] + A3[pk3(p, 2, 2)]) -
               P[20 + p];
        v[1] = e1 * A2[pa];
        v[2] = e1 * A2[pb];
        v[4] = e1 * A2[pc];
        v[3] = e2 * A3[pk3(p, 0, 1)];
        v[5] = e2 * A3[pk3(p, 0, 2)];
        v[6] = e2 * A3[pk3(p, 1, 2)];
        v[7] = 0.0;
        corners8(v);
    }
    const double hc = 0.5 * h;
    const double selfc = self_term ? -G * hc * hc * cube_self_constant() : 0.0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int cl = 2 * (i & 3) + (q & 1) + 8 * (2 * (j & 3) + ((q >> 1) & 1)) + 64 * (2 * (k & 3) + (q >> 2));
        const long long cc = (long long)cn * kCells + cl;
        const long long o = (long long)leaf * kCells + cl;
        double pv = t.loc[cc] + cp[q];
        if (self_term) pv += selfc * rho[o];
        phi[o] = pv;
#pragma unroll
        for (int p = 0; p < 3; p++)
            g[((long long)leaf * 3 + p) * kCells + cl] =
                (t.loc[(20 + p) * N + cc] - t.loc[(1 + p) * N + cc]) - cg[p][q];
    }
}

// FP32-bulk form of k_l2l_leafkids: the shift to the parent's centre and the
// sign-transform corrections at the 8 children (the terms in the offsets) in
// FP32; the parent's coefficients, the children's own expansions and every
// sum in FP64, each FP32 correction widened exactly once.  About 125 FP64
// operations per parent cell instead of 280.
__global__ void __launch_bounds__(64) k_l2l_leafkids_bulk(DevTree t, int first,
                                                          const double* __restrict__ rho,
                                                          double* __restrict__ phi,
                                                          double* __restrict__ g, double G,
                                                          int self_term) {
    const int node = first + (blockIdx.x >> 3);
    const int child0 = t.node_child[node];
    if (child0 < 0) return;
    const long long N = t.n_cells;
    const int c = ((blockIdx.x & 7) << 6) + threadIdx.x;
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int cn = child0 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2);
    const int leaf = t.node_leaf[cn];
    if (leaf < 0) return;  // interior children: k_l2l at the next level
    const int L = t.node_level[node];
    const double h = t.size / (double)(8 << L);
    const float hf = (float)h;
    const long long pcell = (long long)node * kCells + c;
    double P[kLoc];
#pragma unroll
    for (int r = 0; r < kLoc; r++) P[r] = t.loc[r * N + pcell];
    float Q[20];
#pragma unroll
    for (int r = 1; r < 20; r++) Q[r] = (float)P[r];
    // shift from the parent's centre of mass to its cell centre
    const float* mp = t.mom32 + pcell * kMom;
    const float x = -hf * mp[1], y = -hf * mp[2], z = -hf * mp[3];
    const float* L2 = Q + 4;
    const float* L3 = Q + 10;
    const float A2x = fmaf(L2[0], x, fmaf(L2[1], y, L2[2] * z));
    const float A2y = fmaf(L2[1], x, fmaf(L2[3], y, L2[4] * z));
    const float A2z = fmaf(L2[2], x, fmaf(L2[4], y, L2[5] * z));
    const float xx = x * x, yy = y * y, zz = z * z, xy2 = 2.f * x * y, xz2 = 2.f * x * z, yz2 = 2.f * y * z;
    const float B3x = fmaf(L3[0], xx, fmaf(L3[3], yy, fmaf(L3[5], zz, fmaf(L3[1], xy2, fmaf(L3[2], xz2, L3[4] * yz2)))));
    const float B3y = fmaf(L3[1], xx, fmaf(L3[6], yy, fmaf(L3[8], zz, fmaf(L3[3], xy2, fmaf(L3[4], xz2, L3[7] * yz2)))));
    const float B3z = fmaf(L3[2], xx, fmaf(L3[7], yy, fmaf(L3[9], zz, fmaf(L3[4], xy2, fmaf(L3[5], xz2, L3[8] * yz2)))));
    // the shifted expansion A: A0 and A1 as FP64 base plus FP32 correction,
    // A1, A2, A3 also in FP32 for the corner terms
    const double A0 = P[0] + widen(fmaf(Q[1], x, fmaf(Q[2], y, Q[3] * z)) +
                                   0.5f * fmaf(A2x, x, fmaf(A2y, y, A2z * z)) +
                                   (1.0f / 6.0f) * fmaf(B3x, x, fmaf(B3y, y, B3z * z)));
    const float c1[3] = {fmaf(0.5f, B3x, A2x), fmaf(0.5f, B3y, A2y), fmaf(0.5f, B3z, A2z)};
    float A[20];
#pragma unroll
    for (int a = 0; a < 3; a++) A[1 + a] = Q[1 + a] + c1[a];
    A[4] = L2[0] + fmaf(L3[0], x, fmaf(L3[1], y, L3[2] * z));
    A[5] = L2[1] + fmaf(L3[1], x, fmaf(L3[3], y, L3[4] * z));
    A[6] = L2[2] + fmaf(L3[2], x, fmaf(L3[4], y, L3[5] * z));
    A[7] = L2[3] + fmaf(L3[3], x, fmaf(L3[6], y, L3[7] * z));
    A[8] = L2[4] + fmaf(L3[4], x, fmaf(L3[7], y, L3[8] * z));
    A[9] = L2[5] + fmaf(L3[5], x, fmaf(L3[8], y, L3[9] * z));
#pragma unroll
    for (int r = 0; r < 10; r++) A[10 + r] = L3[r];
    const float* A2 = A + 4;
    const float* A3 = A + 10;
    const float e1 = 0.25f * hf, e2 = e1 * e1, e3 = e2 * e1;
    // potential corrections at the 8 corners (A0 added in FP64)
    float cp[8];
    cp[0] = 0.5f * e2 * (A2[0] + A2[3] + A2[5]);
    cp[1] = e1 * A[1] + (e3 / 6.0f) * (A3[0] + 3.0f * (A3[3] + A3[5]));
    cp[2] = e1 * A[2] + (e3 / 6.0f) * (A3[6] + 3.0f * (A3[1] + A3[8]));
    cp[4] = e1 * A[3] + (e3 / 6.0f) * (A3[9] + 3.0f * (A3[2] + A3[7]));
    cp[3] = e2 * A2[1];
    cp[5] = e2 * A2[2];
    cp[6] = e2 * A2[4];
    cp[7] = e3 * A3[4];
    corners8(cp);
    // gradient corrections (the base A1 - a_c(parent) in FP64)
    float cg[3][8];
    double base[3];
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const int pa = p == 0 ? 0 : (p == 1 ? 1 : 2);  // packed (p, x)
        const int pb = p == 0 ? 1 : (p == 1 ? 3 : 4);  // packed (p, y)
        const int pc = p == 0 ? 2 : (p == 1 ? 4 : 5);  // packed (p, z)
        base[p] = (P[1 + p] + widen(c1[p])) - P[20 + p];
        float* v = cg[p];
        v[0] = 0.5f * e2 * (A3[pk3(p, 0, 0)] + A3[pk3(p, 1, 1)] + A3[pk3(p, 2, 2)]);
        v[1] = e1 * A2[pa];
        v[2] = e1 * A2[pb];
        v[4] = e1 * A2[pc];
        v[3] = e2 * A3[pk3(p, 0, 1)];
        v[5] = e2 * A3[pk3(p, 0, 2)];
        v[6] = e2 * A3[pk3(p, 1, 2)];
        v[7] = 0.0f;
        corners8(v);
    }
    const double hc = 0.5 * h;
    const double selfc = self_term ? -G * hc * hc * cube_self_constant() : 0.0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int cl = 2 * (i & 3) + (q & 1) + 8 * (2 * (j & 3) + ((q >> 1) & 1)) + 64 * (2 * (k & 3) + (q >> 2));
        const long long cc = (long long)cn * kCells + cl;
        const long long o = (long long)leaf * kCells + cl;
        double pv = (t.loc[cc] + A0) + widen(cp[q]);
        if (self_term) pv += selfc * rho[o];
        phi[o] = pv;
#pragma unroll
        for (int p = 0; p < 3; p++)
            g[((long long)leaf * 3 + p) * kCells + cl] =
                ((t.loc[(20 + p) * N + cc] - t.loc[(1 + p) * N + cc]) - base[p]) - widen(cg[p][q]);
    }
}

}  // namespace

void launch_l2l(const DevTree& t, int kinds, int first, int count, const double* rho,
                double* phi, double* g, double G, int self_term, int precision, cudaStream_t s) {
    if (count <= 0) return;
    const bool bulk = precision == kPrecWide;  // the FP32-bulk form keeps L2L in FP64
    if (kinds & 1) {
        if (bulk) k_l2l<true><<<count * 16, 32, 0, s>>>(t, first, rho, phi, g, G, self_term);
        else k_l2l<false><<<count * 16, 32, 0, s>>>(t, first, rho, phi, g, G, self_term);
    }
    if (kinds & 2) {
        if (bulk) k_l2l_leafkids_bulk<<<count * 8, 64, 0, s>>>(t, first, rho, phi, g, G, self_term);
        else k_l2l_leafkids<<<count * 8, 64, 0, s>>>(t, first, rho, phi, g, G, self_term);
    }
}

}  // namespace otfmm
