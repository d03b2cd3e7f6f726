// Leaf-leaf pairs of every leaf node of level >= 1: the lattice part of the
// cell-to-cell interactions (stencil approach, Sec. 5.5).
//
// Two leaf cells are point masses at their cell centres, so their pair vector
// is R = -d h exactly and the pair adds m_B (1/|d|, D1(-d)) / (h, h^2) to the
// target's (L0, L1) -- near pairs exactly (the monopole-monopole field) and
// far pairs as the order-3 M2L of two monopoles, which reduces to the same
// two terms at a leaf target.  Over one leaf node this is a small 3-D
// convolution of the masses with a parity-dependent stencil.
//
// A CTA of 8 warps handles one leaf node at a time (one warp per parity
// class of targets, each lane 2 targets 4 cells apart in z).  The masses of the node and of a margin w
// around it are staged once in shared memory (parity-split, padded so a warp
// reads 32 banks); cells of absent or interior neighbours are stored as zero
// mass, so the inner loop has no branches: per stencil entry one broadcast
// load of the table and the halo offset, two shared loads, eight FMAs (the
// near entries in (d, -d) pairs, fewer).
// FP64 form: one kernel, one FP64 halo for every pair.  FP32-bulk form: two
// kernels, far pairs from an FP32 halo with FP32 arithmetic and near pairs
// from an FP64 halo of width floor(1/theta) in FP64; both flushed in FP64.
#include "lattice.hpp"

namespace otfmm {

namespace {

// Fills a parity-split halo of width w with the masses of the leaf cells
// around `node` (zero where there is no leaf cell at this level).  The 27
// neighbours are resolved once into shared memory (s_nbl: the neighbour node
// if it is a leaf, else -1); then one warp per halo row, lanes along x, each
// mass copied by cp.async straight into its halo slot (coalesced reads of
// the contiguous FP64 or FP32 mass array, no conversion, and nothing waits
// per element).  The caller waits (cp.async.wait_all) and synchronises.
__device__ __forceinline__ const double* mass_array(const DevTree& t, double) { return t.mom64; }
__device__ __forceinline__ const float* mass_array(const DevTree& t, float) { return t.m32; }

template <class T>
__device__ __forceinline__ void fill_halo(const DevTree& t, int node, int w, T* halo, int* s_nbl) {
    if (threadIdx.x < 27) {
        const int nb = __ldg(t.nbr + (long long)node * 27 + threadIdx.x);
        s_nbl[threadIdx.x] = nb >= 0 && __ldg(t.node_leaf + nb) >= 0 ? nb : -1;
    }
    __syncthreads();
    const T* __restrict__ mass = mass_array(t, T(0));
    const int hw = 8 + 2 * w;
    const int lane = threadIdx.x & 31;
    const int nwarp = blockDim.x >> 5;
    const int x = lane - w;
    if (lane >= hw) return;
    const int sx = (x >> 3) + 1, lx = x & 7;
    int y = (threadIdx.x >> 5) % hw - w, z = (threadIdx.x >> 5) / hw - w;
    for (int row = threadIdx.x >> 5; row < hw * hw; row += nwarp) {
        const int nb = s_nbl[sx + 3 * ((y >> 3) + 1) + 9 * ((z >> 3) + 1)];
        T* dst = halo + halo_index(x, y, z, w);
        if (nb >= 0)
            cp_async<sizeof(T)>(dst, mass + (long long)nb * kCells + lx + 8 * (y & 7) + 64 * (z & 7));
        else
            *dst = T(0.0);
        y += nwarp;  // next row of this warp: (y, z) advanced without a division
        while (y >= hw - w) {
            y -= hw;
            z++;
        }
    }
}

// Kernel modes: the FP64 form computes every pair from one FP64 halo
// (kAll); the FP32-bulk form splits into an FP64 kernel for the near pairs
// (kNear, halo of width floor(1/theta)) and an FP32 kernel for the far pairs
// (kFar), launched on separate graph branches so that warps of the FP64-pipe
// kernel and of the FP32-pipe kernels share the SMs.
enum LatticeMode { kAll = 0, kNear = 1, kFar = 2 };

// Exact near pairs for the near set 0 < |d|^2 <= 4 (theta = 0.5), unrolled
// with the parity class as a template parameter (near2_code and its
// coefficients are in lattice.hpp): every halo offset is an immediate, the
// coefficients are constants and the zero components of D1 cost nothing --
// 78 FP64 operations per target instead of 96, and no table loads.
template <int PAR, int N>
__device__ __forceinline__ void near2_pairs(const double* hd, int t1, double (&dv)[4], double (&ev)[4]) {
    constexpr int code = near2_code(N);
    constexpr int dx = code % 5 - 2, dy = (code / 5) % 5 - 2, dz = code / 25 - 2;
    constexpr int r2 = dx * dx + dy * dy + dz * dz;
    constexpr int px = PAR & 1, py = (PAR >> 1) & 1, pz = PAR >> 2;
    constexpr int op = halo_index(px + dx, py + dy, pz + dz, 2);
    constexpr int om = halo_index(px - dx, py - dy, pz - dz, 2);
    constexpr int t2 = 2 * halo_pz(2);  // the second target, 4 cells up in z
    constexpr double c0 = near2_inv_r(r2);
    constexpr double cx = dx * near2_inv_r3(r2), cy = dy * near2_inv_r3(r2), cz = dz * near2_inv_r3(r2);
    const double p1 = hd[t1 + op], q1 = hd[t1 + om], p2 = hd[t1 + op + t2], q2 = hd[t1 + om + t2];
    const double s1 = p1 + q1, r1 = p1 - q1, s2 = p2 + q2, r2v = p2 - q2;
    dv[0] = fma(s1, c0, dv[0]);
    ev[0] = fma(s2, c0, ev[0]);
    if (dx != 0) {
        dv[1] = fma(r1, cx, dv[1]);
        ev[1] = fma(r2v, cx, ev[1]);
    }
    if (dy != 0) {
        dv[2] = fma(r1, cy, dv[2]);
        ev[2] = fma(r2v, cy, ev[2]);
    }
    if (dz != 0) {
        dv[3] = fma(r1, cz, dv[3]);
        ev[3] = fma(r2v, cz, ev[3]);
    }
    if constexpr (N + 1 < 16) near2_pairs<PAR, N + 1>(hd, t1, dv, ev);
}

template <int PAR>
__device__ __forceinline__ void near2_all(const double* hd, int t1, double (&dv)[4], double (&ev)[4]) {
    near2_pairs<PAR, 0>(hd, t1, dv, ev);
}

// One node of the lattice pairs, by a CTA of 8 warps (one per parity class).
template <int MODE>
__device__ __forceinline__ void lattice_node(const DevTree& t, const DevPlan& p, const DevLattice& lp,
                                             const LevelScales& sc, int node,
                                             unsigned char* smem, int* s_nbl) {
    const int w = MODE == kNear ? lp.w_near : lp.w_far;
    fill_halo<double>(t, node, w, reinterpret_cast<double*>(smem), s_nbl);
    cp_async_wait_all();
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int par = threadIdx.x >> 5;  // one parity class per warp
    const int a = lane & 3, b = (lane >> 2) & 3, c = lane >> 4;
    const int px = par & 1, py = (par >> 1) & 1, pz = par >> 2;
    const int base = p.list_first[par];
    const int len = p.list_len[par];
    const int t1 = a + kHaloPy * b + halo_pz(w) * c;  // lane offset in the halo
    const int t2 = 2 * halo_pz(w);                     // second target: 4 cells up in z
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;    // FP64 sums, target 1
    double e0 = 0.0, e1 = 0.0, e2 = 0.0, e3 = 0.0;    // FP64 sums, target 2
    if (MODE == kNear && lp.n_near == 32 && w == 2) {
        const double* hd = reinterpret_cast<const double*>(smem);
        double dv[4] = {0.0, 0.0, 0.0, 0.0}, ev[4] = {0.0, 0.0, 0.0, 0.0};
        switch (par) {  // warp-uniform
            case 0: near2_all<0>(hd, t1, dv, ev); break;
            case 1: near2_all<1>(hd, t1, dv, ev); break;
            case 2: near2_all<2>(hd, t1, dv, ev); break;
            case 3: near2_all<3>(hd, t1, dv, ev); break;
            case 4: near2_all<4>(hd, t1, dv, ev); break;
            case 5: near2_all<5>(hd, t1, dv, ev); break;
            case 6: near2_all<6>(hd, t1, dv, ev); break;
            default: near2_all<7>(hd, t1, dv, ev); break;
        }
        d0 = dv[0]; d1 = dv[1]; d2 = dv[2]; d3 = dv[3];
        e0 = ev[0]; e1 = ev[1]; e2 = ev[2]; e3 = ev[3];
    } else if (MODE != kFar) {
        // Near entries come in (d, -d) pairs: entry q and entry n_near - 1 - q
        // (the near set is centrally symmetric and sorted).  With D0 even and
        // D1 odd, a pair costs 6 FP64 operations per target instead of 8:
        //   L0 += D0(d) (m(t+d) + m(t-d)),  L1 += D1(d) (m(t+d) - m(t-d)).
        const double* hd = reinterpret_cast<const double*>(smem);
        const int* hn = MODE == kNear ? lp.hoff_near : lp.hoff_far;
        const int npair = lp.n_near >> 1;
#pragma unroll 2
        for (int q = 0; q < npair; q++) {
            const int o1 = __ldg(hn + base + q) + t1;
            const int o2 = __ldg(hn + base + lp.n_near - 1 - q) + t1;
            const double2 k0 = __ldg(p.tab64 + 2 * (base + q)), k1 = __ldg(p.tab64 + 2 * (base + q) + 1);
            const double p1 = hd[o1], q1 = hd[o2], p2 = hd[o1 + t2], q2 = hd[o2 + t2];
            const double s1 = p1 + q1, r1 = p1 - q1, s2 = p2 + q2, r2 = p2 - q2;
            d0 = fma(s1, k0.x, d0); d1 = fma(r1, k0.y, d1); d2 = fma(r1, k1.x, d2); d3 = fma(r1, k1.y, d3);
            e0 = fma(s2, k0.x, e0); e1 = fma(r2, k0.y, e1); e2 = fma(r2, k1.x, e2); e3 = fma(r2, k1.y, e3);
        }
    }
    if (MODE == kAll) {
        const double* hd = reinterpret_cast<const double*>(smem);
#pragma unroll 4
        for (int q = lp.n_near; q < len; q++) {
            const int o = __ldg(lp.hoff_far + base + q) + t1;
            const double2 k0 = __ldg(p.tab64 + 2 * (base + q)), k1 = __ldg(p.tab64 + 2 * (base + q) + 1);
            const double m1 = hd[o], m2 = hd[o + t2];
            d0 = fma(m1, k0.x, d0); d1 = fma(m1, k0.y, d1); d2 = fma(m1, k1.x, d2); d3 = fma(m1, k1.y, d3);
            e0 = fma(m2, k0.x, e0); e1 = fma(m2, k0.y, e1); e2 = fma(m2, k1.x, e2); e3 = fma(m2, k1.y, e3);
        }
    }
    // to physical units: L0 * (-G / h), L1 * (-G / h^2)
    const int L = t.node_level[node];
    const double s1 = sc.s64[L][0], s2 = sc.s64[L][1];
    const long long N = t.n_cells;
    const long long c1 = (long long)node * kCells + (2 * a + px) + 8 * (2 * b + py) + 64 * (2 * c + pz);
    const long long c2 = c1 + 256;
    double* loc = t.loc;
    atomicAdd(loc + c1, s1 * d0);
    atomicAdd(loc + N + c1, s2 * d1);
    atomicAdd(loc + 2 * N + c1, s2 * d2);
    atomicAdd(loc + 3 * N + c1, s2 * d3);
    atomicAdd(loc + c2, s1 * e0);
    atomicAdd(loc + N + c2, s2 * e1);
    atomicAdd(loc + 2 * N + c2, s2 * e2);
    atomicAdd(loc + 3 * N + c2, s2 * e3);
}

// Shared-memory layout of the FP32 far kernel: the FP32 halo, then (when it
// fits) the far part of the 8 parity lists: coefficients float4 [8][n_far_max],
// halo offsets int [8][n_far_max].
__device__ __forceinline__ float4* far_coef(unsigned char* smem, const DevLattice& lp) {
    return reinterpret_cast<float4*>(smem + sizeof(float) * 8 * (size_t)halo_sub(lp.w_far));
}
__device__ __forceinline__ int* far_hoff(unsigned char* smem, const DevLattice& lp) {
    return reinterpret_cast<int*>(far_coef(smem, lp) + 8 * lp.n_far_max);
}

// Copies the far tables into shared memory (once per persistent CTA).
__device__ __forceinline__ void lattice_far_tables(const DevPlan& p, const DevLattice& lp,
                                                   unsigned char* smem) {
    float4* kc = far_coef(smem, lp);
    int* ho = far_hoff(smem, lp);
    for (int par = 0; par < 8; par++) {
        const int len = p.list_len[par] - lp.n_near;
        const int at = p.list_first[par] + lp.n_near;
        for (int q = threadIdx.x; q < len; q += blockDim.x) {
            cp_async<16>(kc + par * lp.n_far_max + q, p.tab32 + at + q);
            cp_async<4>(ho + par * lp.n_far_max + q, lp.hoff_far + at + q);
        }
    }
    cp_async_wait_all();  // made visible to the CTA by the caller's next barrier
}

// FP32 far pairs of one node by a CTA of 4 warps: a half-warp per parity
// class, each lane 4 targets along z (so one table entry feeds 16 FMAs);
// FP32 sums widened exactly to FP64 once per target.
__device__ __forceinline__ void lattice_far_node(const DevTree& t, const DevPlan& p,
                                                 const DevLattice& lp, const LevelScales& sc,
                                                 int node, unsigned char* smem, int* s_nbl) {
    const int w = lp.w_far;
    fill_halo<float>(t, node, w, reinterpret_cast<float*>(smem), s_nbl);
    cp_async_wait_all();
    __syncthreads();
    const float* hf = reinterpret_cast<const float*>(smem);
    const int lane = threadIdx.x & 31;
    const int par = 2 * (threadIdx.x >> 5) + (lane >> 4);
    const int a = lane & 3, b = (lane >> 2) & 3;
    const int px = par & 1, py = (par >> 1) & 1, pz = par >> 2;
    const int base = p.list_first[par];
    const int len = p.list_len[par];
    const int pzs = halo_pz(w);              // z stride of a parity sub-halo
    const int t0 = a + kHaloPy * b;          // lane offset (first target) in the halo
    float f[4][4];
#pragma unroll
    for (int c = 0; c < 4; c++)
#pragma unroll
        for (int r = 0; r < 4; r++) f[c][r] = 0.f;
    auto entry = [&](int o, const float4 k) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const float m = hf[o + c * pzs];
            f[c][0] = fmaf(m, k.x, f[c][0]);
            f[c][1] = fmaf(m, k.y, f[c][1]);
            f[c][2] = fmaf(m, k.z, f[c][2]);
            f[c][3] = fmaf(m, k.w, f[c][3]);
        }
    };
    if (lp.far_table_smem) {
        // tables staged in shared memory by the CTA (lattice_far_tables)
        const float4* kc = far_coef(smem, lp) + par * lp.n_far_max;
        const int* ho = far_hoff(smem, lp) + par * lp.n_far_max;
        const int nf = len - lp.n_near;
#pragma unroll 4
        for (int q = 0; q < nf; q++) entry(ho[q] + t0, kc[q]);
    } else {
#pragma unroll 2
        for (int q = lp.n_near; q < len; q++) entry(__ldg(lp.hoff_far + base + q) + t0, __ldg(p.tab32 + base + q));
    }
    const int L = t.node_level[node];
    const double s1 = sc.s64[L][0], s2 = sc.s64[L][1];
    const long long N = t.n_cells;
    double* loc = t.loc;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const long long cell = (long long)node * kCells + (2 * a + px) + 8 * (2 * b + py) + 64 * (2 * c + pz);
        atomicAdd(loc + cell, s1 * widen(f[c][0]));
        atomicAdd(loc + N + cell, s2 * widen(f[c][1]));
        atomicAdd(loc + 2 * N + cell, s2 * widen(f[c][2]));
        atomicAdd(loc + 3 * N + cell, s2 * widen(f[c][3]));
    }
}

// Persistent CTAs: each takes the next node from its mode's counter until
// none are left, so a bounded number of CTAs per SM leaves room for the
// kernels of the other graph branches on the same SMs.
template <int MODE>
__global__ void __launch_bounds__(256) k_lattice(DevTree t, DevPlan p, DevLattice lp, LevelScales sc) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_task;
    __shared__ int s_nbl[27];
    int* counter = lp.counter + (MODE == kFar ? 1 : 0);
    if (MODE == kFar && lp.far_table_smem) lattice_far_tables(p, lp, smem);  // visible after the next barrier
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(counter, 1);
        __syncthreads();
        const int task = s_task;
        if (task >= lp.n_nodes) break;
        if (MODE == kFar)
            lattice_far_node(t, p, lp, sc, lp.nodes[task], smem, s_nbl);
        else
            lattice_node<MODE>(t, p, lp, sc, lp.nodes[task], smem, s_nbl);
        __syncthreads();  // the halo and s_task are rewritten for the next node
    }
}

}  // namespace

size_t lattice_smem_bytes(int mode, int w_far, int w_near, int far_table_entries) {
    if (mode == kFar)
        return sizeof(float) * 8 * (size_t)halo_sub(w_far) + (size_t)far_table_entries * (16 + 4);
    if (mode == kNear) return sizeof(double) * 8 * (size_t)halo_sub(w_near);
    return sizeof(double) * 8 * (size_t)halo_sub(w_far);
}

void lattice_far_table_plan(DevLattice& lp, const int* list_len) {
    int m = 0;
    for (int par = 0; par < 8; par++) m = list_len[par] - lp.n_near > m ? list_len[par] - lp.n_near : m;
    lp.n_far_max = m;
    lp.far_table_smem = lattice_smem_bytes(kFar, lp.w_far, lp.w_near, 8 * m) <= kLatticeSmemMax ? 1 : 0;
}

// The lattice kernels run as concurrent graph branches; an SM's shared-memory
// carveout is set for the kernel whose CTA it takes first, and a CTA of
// another kernel needing more than that carveout leaves cannot join it.  The
// lattice kernels therefore all ask for the largest carveout (near and far
// pairs then overlap: 158 -> 104 us on the level-3 binary).
template <class K> static bool configure_one(K kernel, int smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
}

int configure_lattice() {
    const int bytes = (int)kLatticeSmemMax;
    if (!configure_one(k_lattice<kAll>, bytes) || !configure_one(k_lattice<kNear>, bytes) ||
        !configure_one(k_lattice<kFar>, bytes)) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}

void launch_lattice(const DevTree& t, const DevPlan& p, const DevLattice& lp, int precision,
                    double G, int ctas, cudaStream_t s, cudaStream_t s_far) {
    if (lp.n_nodes <= 0) return;
    const LevelScales sc = level_scales(t.inv_side8, G);
    const int grid = ctas > 0 && ctas < lp.n_nodes ? ctas : lp.n_nodes;
    if (precision == kPrecWide) {
        const int tab = lp.far_table_smem ? 8 * lp.n_far_max : 0;
        cudaStream_t sf = s_far ? s_far : s;
        k_lattice<kNear><<<grid, 256, lattice_smem_bytes(kNear, lp.w_far, lp.w_near, 0), s>>>(t, p, lp, sc);
        k_lattice<kFar><<<grid, 128, lattice_smem_bytes(kFar, lp.w_far, lp.w_near, tab), sf>>>(t, p, lp, sc);
    } else {
        k_lattice<kAll><<<grid, 256, lattice_smem_bytes(kAll, lp.w_far, lp.w_near, 0), s>>>(t, p, lp, sc);
    }
}

}  // namespace otfmm
