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
// One CTA per leaf node, 8 warps (one per parity class of targets), each lane
// 2 targets 4 cells apart in z.  The masses of the node and of a margin w
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
// around `node` (zero where there is no leaf cell at this level): one warp
// per row of the halo, lanes along x.  The masses are read from the
// contiguous FP64 or FP32 array (coalesced), so no conversion is needed.
__device__ __forceinline__ const double* mass_array(const DevTree& t, double) { return t.mom64; }
__device__ __forceinline__ const float* mass_array(const DevTree& t, float) { return t.m32; }

template <class T>
__device__ __forceinline__ void fill_halo(const DevTree& t, int node, int w, T* halo) {
    const T* __restrict__ mass = mass_array(t, T(0));
    const int hw = 8 + 2 * w;
    const int* nbr = t.nbr + (long long)node * 27;
    const int lane = threadIdx.x & 31;
    const int nwarp = blockDim.x >> 5;
    for (int row = threadIdx.x >> 5; row < hw * hw; row += nwarp) {
        const int y = row % hw - w, z = row / hw - w;
        const int x = lane - w;
        if (lane >= hw) continue;
        const int slot = ((x >> 3) + 1) + 3 * ((y >> 3) + 1) + 9 * ((z >> 3) + 1);
        const int nb = __ldg(nbr + slot);
        T v = T(0.0);
        if (nb >= 0 && __ldg(t.node_leaf + nb) >= 0)
            v = mass[(long long)nb * kCells + (x & 7) + 8 * (y & 7) + 64 * (z & 7)];
        halo[halo_index(x, y, z, w)] = v;
    }
}

// Kernel modes: the FP64 form computes every pair from one FP64 halo
// (kAll); the FP32-bulk form splits into an FP64 kernel for the near pairs
// (kNear, halo of width floor(1/theta)) and an FP32 kernel for the far pairs
// (kFar), launched on separate graph branches so that warps of the FP64-pipe
// kernel and of the FP32-pipe kernels share the SMs.
enum LatticeMode { kAll = 0, kNear = 1, kFar = 2 };

template <int MODE>
__global__ void __launch_bounds__(256) k_lattice(DevTree t, DevPlan p, DevLattice lp, LevelScales sc) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int node = lp.nodes[blockIdx.x];
    const int w = MODE == kNear ? lp.w_near : lp.w_far;
    if (MODE == kFar)
        fill_halo<float>(t, node, w, reinterpret_cast<float*>(smem));
    else
        fill_halo<double>(t, node, w, reinterpret_cast<double*>(smem));
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
    if (MODE != kFar) {
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
    if (MODE == kFar) {
        // far pairs in FP32, widened exactly to FP64 once per target
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
        const float* hf = reinterpret_cast<const float*>(smem);
#pragma unroll 4
        for (int q = lp.n_near; q < len; q++) {
            const int o = __ldg(lp.hoff_far + base + q) + t1;
            const float4 k = __ldg(p.tab32 + base + q);
            const float m1 = hf[o], m2 = hf[o + t2];
            f0 = fmaf(m1, k.x, f0); f1 = fmaf(m1, k.y, f1); f2 = fmaf(m1, k.z, f2); f3 = fmaf(m1, k.w, f3);
            g0 = fmaf(m2, k.x, g0); g1 = fmaf(m2, k.y, g1); g2 = fmaf(m2, k.z, g2); g3 = fmaf(m2, k.w, g3);
        }
        d0 = widen(f0); d1 = widen(f1); d2 = widen(f2); d3 = widen(f3);
        e0 = widen(g0); e1 = widen(g1); e2 = widen(g2); e3 = widen(g3);
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

}  // namespace

size_t lattice_smem_bytes(int mode, int w_far, int w_near) {
    if (mode == kFar) return sizeof(float) * 8 * (size_t)halo_sub(w_far);
    if (mode == kNear) return sizeof(double) * 8 * (size_t)halo_sub(w_near);
    return sizeof(double) * 8 * (size_t)halo_sub(w_far);
}

int configure_lattice() {
    const int bytes = 160 * 1024;
    if (cudaFuncSetAttribute(k_lattice<kAll>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_lattice<kNear>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_lattice<kFar>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}

void launch_lattice(const DevTree& t, const DevPlan& p, const DevLattice& lp, int precision,
                    double G, cudaStream_t s, cudaStream_t s_far) {
    if (lp.n_nodes <= 0) return;
    const LevelScales sc = level_scales(t.inv_side8, G);
    if (precision == 1) {
        k_lattice<kNear><<<lp.n_nodes, 256, lattice_smem_bytes(kNear, lp.w_far, lp.w_near), s>>>(t, p, lp, sc);
        k_lattice<kFar><<<lp.n_nodes, 256, lattice_smem_bytes(kFar, lp.w_far, lp.w_near),
                          s_far ? s_far : s>>>(t, p, lp, sc);
    } else {
        k_lattice<kAll><<<lp.n_nodes, 256, lattice_smem_bytes(kAll, lp.w_far, lp.w_near), s>>>(t, p, lp, sc);
    }
}

}  // namespace otfmm
