// Upward pass of the FMM gravity solve on GB300: leaf masses and exact M2M.
//
// A leaf cell is a point mass m = rho h^3 at its centre (its offset dX,
// M2 and M3 are zero and are written once when the tree is built).  An
// interior cell's moments are the exact moments of its 8 children about the
// parent's centre of mass (multipole moments up to order 3, implied by the
// FMM of Sec. 4.3.2).  Everything is FP64; an FP32 copy is written for the
// FP32-bulk interaction form.  Both kernels also zero the expansions of their
// cells, which the interaction kernels then accumulate into.
//
// M2M of cells with interior children uses 8 threads per parent cell, one
// per child: the children's masses and mass-weighted positions are summed by
// warp shuffles, every lane forms its child's contribution about the common
// centre of mass, and a reduce-scatter leaves each lane with the sums of the
// record entries it writes.  One warp per block, so the coarse levels (1 node
// at level 0, 8 at level 1) still spread over many SMs of the FP64 pipe.  Cells whose
// children are leaves (the most numerous) take a cheaper path: their children
// sit at fixed offsets, so the moments are signed sums of 8 masses.
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
    const long long N = t.n_cells;
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
        const double m = rho[(long long)leaf * kCells + c] * h3;
        const long long cell = (long long)node * kCells + c;
        t.mom64[cell] = m;
        t.rec64[cell * kRec] = m;
        t.mom32[cell * kMom] = (float)m;
        t.m32[cell] = (float)m;
        // a leaf cell's expansion: L0, L1 and the correction acceleration
        t.loc[cell] = 0.0;
        t.loc[N + cell] = 0.0;
        t.loc[2 * N + cell] = 0.0;
        t.loc[3 * N + cell] = 0.0;
        t.loc[20 * N + cell] = 0.0;
        t.loc[21 * N + cell] = 0.0;
        t.loc[22 * N + cell] = 0.0;
    }
}

// Packed symmetric tensors (rank 2: xx xy xz yy yz zz; rank 3: xxx xxy xxz
// xyy xyz xzz yyy yyz yzz zzz), written out component by component so that
// nothing is indexed at run time.
// o = s u v (rank 2, u v symmetric in use: u = s' v)
template <class T> __device__ __forceinline__ void outer2(T s, const T* v, T* o) {
    o[0] = s * v[0] * v[0]; o[1] = s * v[0] * v[1]; o[2] = s * v[0] * v[2];
    o[3] = s * v[1] * v[1]; o[4] = s * v[1] * v[2]; o[5] = s * v[2] * v[2];
}
// o = s v v v (rank 3)
template <class T> __device__ __forceinline__ void outer3(T s, const T* v, T* o) {
    const T xx = s * v[0] * v[0], yy = s * v[1] * v[1], zz = s * v[2] * v[2];
    o[0] = xx * v[0]; o[1] = xx * v[1]; o[2] = xx * v[2]; o[3] = yy * v[0];
    o[4] = s * v[0] * v[1] * v[2]; o[5] = zz * v[0]; o[6] = yy * v[1]; o[7] = yy * v[2];
    o[8] = zz * v[1]; o[9] = zz * v[2];
}
// o_ijk = P_ij v_k + P_ik v_j + P_jk v_i for a packed symmetric rank-2 P
template <class T> __device__ __forceinline__ void sym3_of(const T* P, const T* v, T* o) {
    o[0] = T(3) * P[0] * v[0];
    o[1] = P[0] * v[1] + T(2) * P[1] * v[0];
    o[2] = P[0] * v[2] + T(2) * P[2] * v[0];
    o[3] = T(2) * P[1] * v[1] + P[3] * v[0];
    o[4] = P[1] * v[2] + P[2] * v[1] + P[4] * v[0];
    o[5] = T(2) * P[2] * v[2] + P[5] * v[0];
    o[6] = T(3) * P[3] * v[1];
    o[7] = P[3] * v[2] + T(2) * P[4] * v[1];
    o[8] = T(2) * P[4] * v[2] + P[5] * v[1];
    o[9] = T(3) * P[5] * v[2];
}

// sum over the 8 lanes of a parent cell (lanes 8g .. 8g+7 of a warp)
__device__ __forceinline__ double sum8(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}

// Butterfly step of a reduce-scatter over lanes q and q ^ mask: a lane keeps
// the component of each pair (lo, hi) on its own side of the mask bit, adds
// its partner's copy of it, and hands over the other one.
__device__ __forceinline__ double keep_add(bool upper, double lo, double hi, int mask) {
    const double keep = upper ? hi : lo;
    const double give = upper ? lo : hi;
    return keep + __shfl_xor_sync(0xffffffffu, give, mask);
}

// One warp per block = 4 parent cells x 8 children; 128 blocks per node, so
// that the single node of level 0 already spreads over 128 SMs.  Cells whose
// children are leaf cells are left to k_m2m_leafkids; the 4 cells of a warp
// share one child node, so that test is uniform per warp.  BULK (FP32-bulk
// form): the products of the shift (m d d, sym(M2 d), m d d d) in FP32, each
// widened exactly and added to the FP64 sums; masses, centres of mass and
// every sum stay FP64.
template <bool BULK>
__global__ void __launch_bounds__(32) k_m2m(DevTree t, int first) {
    const int node = first + (blockIdx.x >> 7);
    const int child0 = t.node_child[node];
    if (child0 < 0) return;  // leaf node: moments come from rho
    const long long N = t.n_cells;
    const int c = ((blockIdx.x & 127) << 2) + (threadIdx.x >> 3);  // parent cell in the node
    const int q = threadIdx.x & 7;                                  // child octant
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int a = q & 1, b = (q >> 1) & 1, e = q >> 2;
    // the 8 children of cell (i, j, k) lie in child node (i>>2, j>>2, k>>2)
    const int cn = child0 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2);
    if (t.node_child[cn] < 0) return;  // leaf children: k_m2m_leafkids
    const long long cc = (long long)cn * kCells + (2 * (i & 3) + a) + 8 * (2 * (j & 3) + b) +
                         64 * (2 * (k & 3) + e);
    const double m = t.mom64[cc];
    // child centre of mass relative to the parent cell centre, parent units
    double pos[3];
    pos[0] = 0.5 * ((a - 0.5) + t.mom64[N + cc]);
    pos[1] = 0.5 * ((b - 0.5) + t.mom64[2 * N + cc]);
    pos[2] = 0.5 * ((e - 0.5) + t.mom64[3 * N + cc]);
    const double M = sum8(m);
    double X[3];
#pragma unroll
    for (int s = 0; s < 3; s++) X[s] = sum8(m * pos[s]);  // shuffles: every lane takes part
    const double iM = M != 0.0 ? 1.0 / M : 0.0;               // zero mass: moments about the centre
#pragma unroll
    for (int s = 0; s < 3; s++) X[s] *= iM;
    // the child's shifted moments: M2 + m d d, M3 + sym(M2 d) + m d d d
    double S[16];
    if (BULK) {
        const float* mc = t.mom32 + cc * kMom;
        const float dfv[3] = {0.5f * (((float)a - 0.5f) + mc[1]) - (float)X[0],
                              0.5f * (((float)b - 0.5f) + mc[2]) - (float)X[1],
                              0.5f * (((float)e - 0.5f) + mc[3]) - (float)X[2]};
        float c2[6], p2[6], p3[10], t3[10];
#pragma unroll
        for (int r = 0; r < 6; r++) c2[r] = 0.25f * mc[4 + r];  // child units -> parent
        outer2(mc[0], dfv, p2);
        outer3(mc[0], dfv, p3);
        sym3_of(c2, dfv, t3);
#pragma unroll
        for (int r = 0; r < 6; r++) S[r] = fma(0.25, t.mom64[(4 + r) * N + cc], widen(p2[r]));
#pragma unroll
        for (int r = 0; r < 10; r++) S[6 + r] = fma(0.125, t.mom64[(10 + r) * N + cc], widen(p3[r] + t3[r]));
    } else {
        const double d[3] = {pos[0] - X[0], pos[1] - X[1], pos[2] - X[2]};
        double c2[6], t3[10];
#pragma unroll
        for (int r = 0; r < 6; r++) c2[r] = 0.25 * t.mom64[(4 + r) * N + cc];  // child units -> parent
        outer2(m, d, S);
#pragma unroll
        for (int r = 0; r < 6; r++) S[r] += c2[r];
        outer3(m, d, S + 6);
        sym3_of(c2, d, t3);
#pragma unroll
        for (int r = 0; r < 10; r++) S[6 + r] += 0.125 * t.mom64[(10 + r) * N + cc] + t3[r];
    }
    // the traces are linear in the moments: M3 trace vector t_i = M3_ijj
    // (packed xxx+xyy+xzz, xxy+yyy+yzz, xxz+yyz+zzz) and trace(M2)
    const double T[4] = {S[6] + S[9] + S[11], S[7] + S[12] + S[14], S[8] + S[13] + S[15],
                         S[0] + S[3] + S[5]};
    // reduce-scatter over the 8 lanes: lane q ends with the sums of S[q] and
    // S[q + 8] (record entries 4 + q and 12 + q) and of T[q >> 1]
    const bool u4 = q & 4, u2 = q & 2, u1 = q & 1;
    double R8[8], R4[4], R2[2];
#pragma unroll
    for (int h = 0; h < 8; h++) {
        const int lo = (h & 3) | ((h & 4) << 1);  // components with bit 2 clear
        R8[h] = keep_add(u4, S[lo], S[lo | 4], 4);
    }
#pragma unroll
    for (int h = 0; h < 4; h++) {
        const int lo = (h & 1) | ((h & 2) << 1);
        R4[h] = keep_add(u2, R8[lo], R8[lo | 2], 2);
    }
#pragma unroll
    for (int h = 0; h < 2; h++) R2[h] = keep_add(u1, R4[2 * h], R4[2 * h + 1], 1);
    const double U0 = keep_add(u4, T[0], T[2], 4);
    const double U1 = keep_add(u4, T[1], T[3], 4);
    double V = keep_add(u2, U0, U1, 2);
    V += __shfl_xor_sync(0xffffffffu, V, 1);
    // each lane writes the record entries it owns: 20 moments (+ the two
    // traces) and 23 zeroed expansions
    const long long cell = (long long)node * kCells + c;
    double* rec = t.rec64 + cell * kRec;
    float* m32 = t.mom32 + cell * kMom;
    rec[4 + q] = R2[0];
    rec[12 + q] = R2[1];
    t.mom64[(4 + q) * N + cell] = R2[0];
    t.mom64[(12 + q) * N + cell] = R2[1];
    m32[4 + q] = (float)R2[0];
    m32[12 + q] = (float)R2[1];
    if (q < 4) {
        const double v = q == 0 ? M : (q == 1 ? X[0] : (q == 2 ? X[1] : X[2]));
        rec[q] = v;
        t.mom64[q * N + cell] = v;
        m32[q] = (float)v;
    }
    if (!u1) rec[20 + (q >> 1)] = V;
    // FP32 octupole per unit mass (M3 / m, entries 10..19, and its trace
    // vector, 20..22) for the correction's target term, the division done
    // here in FP64; entries 13..15 are zero
    float* o32 = t.oct32 + cell * kOct;
    o32[2 + q] = (float)(R2[1] * iM);
    if (q >= 6) o32[q - 6] = (float)(R2[0] * iM);
    if (!u1) o32[10 + (q >> 1)] = q < 6 ? (float)(V * iM) : 0.f;
    if (q == 1 || q == 3) o32[14 + (q >> 1)] = 0.f;
#pragma unroll
    for (int r = q; r < kLoc; r += 8) t.loc[r * N + cell] = 0.0;
}

// In-place Walsh transform of 8 values indexed by octant bits (x = bit 0):
// on return w[q] = sum_k v[k] (-1)^popcount(q & k).
__device__ __forceinline__ void walsh8(double* w) {
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (!(q & bit)) {
                const double u = w[q], v = w[q | bit];
                w[q] = u + v;
                w[q | bit] = u - v;
            }
}

// M2M of a cell whose 8 children are leaf cells: point masses at offsets
// s/4 (s in {-1, 1}^3, parent units) from the parent centre, with no offset
// or higher moment of their own.  Their moments about the parent centre are
// signed sums of the masses (a Walsh transform); the parallel-axis shift to
// the centre of mass X gives
//   M2 = P2 - M X X,   M3 = P3 - 3 sym(X P2) + 2 M X X X.
// One thread per parent cell, 8 blocks of 64 per node.  BULK: the
// parallel-axis products in FP32, widened exactly into the FP64 sums.
template <bool BULK>
__global__ void __launch_bounds__(64) k_m2m_leafkids(DevTree t, int first) {
    const int node = first + (blockIdx.x >> 3);
    const int child0 = t.node_child[node];
    if (child0 < 0) return;
    const long long N = t.n_cells;
    const int c = ((blockIdx.x & 7) << 6) + threadIdx.x;
    const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
    const int cn = child0 + (i >> 2) + 2 * (j >> 2) + 4 * (k >> 2);
    if (t.node_child[cn] >= 0) return;  // interior children: k_m2m
    const long long cbase = (long long)cn * kCells + 2 * (i & 3) + 16 * (j & 3) + 128 * (k & 3);
    double w[8];
#pragma unroll
    for (int q = 0; q < 8; q++) w[q] = t.mom64[cbase + (q & 1) + 8 * ((q >> 1) & 1) + 64 * (q >> 2)];
    walsh8(w);
    // sums of m s_x, m s_y, ... (s = 2 bit - 1, so a bit set counts +)
    const double M = w[0];
    const double Sx = -w[1], Sy = -w[2], Sz = -w[4];
    const double Sxy = w[3], Sxz = w[5], Syz = w[6], Sxyz = -w[7];
    const double iM = M != 0.0 ? 1.0 / M : 0.0;  // zero mass: moments about the centre
    const double X[3] = {0.25 * Sx * iM, 0.25 * Sy * iM, 0.25 * Sz * iM};
    // raw moments about the parent centre (packed xx xy xz yy yz zz, ...)
    const double P2[6] = {0.0625 * M, 0.0625 * Sxy, 0.0625 * Sxz, 0.0625 * M, 0.0625 * Syz, 0.0625 * M};
    const double s64 = 1.0 / 64.0;
    const double P3[10] = {s64 * Sx, s64 * Sy, s64 * Sz, s64 * Sx, s64 * Sxyz,
                           s64 * Sx, s64 * Sy, s64 * Sz, s64 * Sy, s64 * Sz};
    double S2[6], S3[10];
    // parallel-axis shift to the centre of mass: M2 = P2 - M X X,
    // M3 = P3 - sym(P2 X) + 2 M X X X
    if (BULK) {
        const float Mf = (float)M;
        const float Xf[3] = {(float)X[0], (float)X[1], (float)X[2]};
        const float P2f[6] = {0.0625f * Mf, 0.0625f * (float)Sxy, 0.0625f * (float)Sxz,
                              0.0625f * Mf, 0.0625f * (float)Syz, 0.0625f * Mf};
        float xx2[6], xxx3[10], px3[10];
        outer2(Mf, Xf, xx2);
        outer3(2.0f * Mf, Xf, xxx3);
        sym3_of(P2f, Xf, px3);
#pragma unroll
        for (int r = 0; r < 6; r++) S2[r] = P2[r] - widen(xx2[r]);
#pragma unroll
        for (int r = 0; r < 10; r++) S3[r] = P3[r] + widen(xxx3[r] - px3[r]);
    } else {
        double xx2[6], xxx3[10], px3[10];
        outer2(M, X, xx2);
        outer3(2.0 * M, X, xxx3);
        sym3_of(P2, X, px3);
#pragma unroll
        for (int r = 0; r < 6; r++) S2[r] = P2[r] - xx2[r];
#pragma unroll
        for (int r = 0; r < 10; r++) S3[r] = P3[r] - px3[r] + xxx3[r];
    }
    const long long cell = (long long)node * kCells + c;
    double v[kRec];
    v[0] = M;
#pragma unroll
    for (int s = 0; s < 3; s++) v[1 + s] = X[s];
#pragma unroll
    for (int r = 0; r < 6; r++) v[4 + r] = S2[r];
#pragma unroll
    for (int r = 0; r < 10; r++) v[10 + r] = S3[r];
    v[20] = S3[0] + S3[3] + S3[5];
    v[21] = S3[1] + S3[6] + S3[8];
    v[22] = S3[2] + S3[7] + S3[9];
    v[23] = S2[0] + S2[3] + S2[5];
#pragma unroll
    for (int r = 0; r < kMom; r++) t.mom64[r * N + cell] = v[r];
    double2* r64 = reinterpret_cast<double2*>(t.rec64 + cell * kRec);
    float4* r32 = reinterpret_cast<float4*>(t.mom32 + cell * kMom);
#pragma unroll
    for (int r = 0; r < kRec / 2; r++) r64[r] = make_double2(v[2 * r], v[2 * r + 1]);
#pragma unroll
    for (int r = 0; r < kMom / 4; r++)
        r32[r] = make_float4((float)v[4 * r], (float)v[4 * r + 1], (float)v[4 * r + 2], (float)v[4 * r + 3]);
    // FP32 octupole per unit mass: M3 / m (v[10..19]) and its trace vector (v[20..22])
    float4* o32 = reinterpret_cast<float4*>(t.oct32 + cell * kOct);
    o32[0] = make_float4((float)(v[10] * iM), (float)(v[11] * iM), (float)(v[12] * iM), (float)(v[13] * iM));
    o32[1] = make_float4((float)(v[14] * iM), (float)(v[15] * iM), (float)(v[16] * iM), (float)(v[17] * iM));
    o32[2] = make_float4((float)(v[18] * iM), (float)(v[19] * iM), (float)(v[20] * iM), (float)(v[21] * iM));
    o32[3] = make_float4((float)(v[22] * iM), 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kLoc; r++) t.loc[r * N + cell] = 0.0;
}

// The moments of one level in physical units, for reading them back: per
// node of the level, component-major [20][512]: m, the centre of mass X,
// M2 h^2 and M3 h^3 (the workspace keeps dX = X - cell centre and the
// moments in units of the cell side h).
__global__ void __launch_bounds__(256) k_get_moments(DevTree t, int first, double* __restrict__ out) {
    const int node = first + blockIdx.x;
    const int L = t.node_level[node];
    const double h = t.size / (double)(8 << L);
    const double h2 = h * h, h3 = h2 * h;
    const int nx = t.node_xyz[3 * node], ny = t.node_xyz[3 * node + 1], nz = t.node_xyz[3 * node + 2];
    const long long N = t.n_cells;
    double* o = out + (long long)blockIdx.x * kMom * kCells;
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
        const long long cell = (long long)node * kCells + c;
        const int ijk[3] = {8 * nx + (c & 7), 8 * ny + ((c >> 3) & 7), 8 * nz + (c >> 6)};
        o[c] = t.mom64[cell];
#pragma unroll
        for (int a = 0; a < 3; a++)
            o[(1 + a) * kCells + c] = t.origin[a] + ((ijk[a] + 0.5) + t.mom64[(1 + a) * N + cell]) * h;
#pragma unroll
        for (int r = 4; r < 10; r++) o[r * kCells + c] = t.mom64[r * N + cell] * h2;
#pragma unroll
        for (int r = 10; r < kMom; r++) o[r * kCells + c] = t.mom64[r * N + cell] * h3;
    }
}

}  // namespace

void launch_get_moments(const DevTree& t, int first, int count, double* out, cudaStream_t s) {
    if (count > 0) k_get_moments<<<count, 256, 0, s>>>(t, first, out);
}

void launch_leaf_moments(const DevTree& t, const int* leaf_node, const double* rho,
                         cudaStream_t s) {
    k_leaf_moments<<<t.n_leaf, 256, 0, s>>>(t, leaf_node, rho);
}

void launch_m2m(const DevTree& t, int kinds, int first, int count, int precision, cudaStream_t s) {
    if (count <= 0) return;
    const bool bulk = precision == kPrecWide;  // the FP32-bulk form keeps M2M in FP64
    if (kinds & 1) {
        if (bulk) k_m2m<true><<<count * 128, 32, 0, s>>>(t, first);
        else k_m2m<false><<<count * 128, 32, 0, s>>>(t, first);
    }
    if (kinds & 2) {
        if (bulk) k_m2m_leafkids<true><<<count * 8, 64, 0, s>>>(t, first);
        else k_m2m_leafkids<false><<<count * 8, 64, 0, s>>>(t, first);
    }
}

}  // namespace otfmm
