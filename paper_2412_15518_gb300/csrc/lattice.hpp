// Launcher of the lattice kernel (lattice.cu): leaf-leaf pairs of the leaf
// nodes of level >= 1.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "common.cuh"

namespace otfmm {

// The near set 0 < |d|^2 <= 4 (theta = 0.5) as 16 pairs (d, -d): the
// representative d of pair n, packed (dx+2) + 5 (dy+2) + 25 (dz+2), and by
// |d|^2 the factors 1/|d| (D0) and 1/|d|^3 (D1 = d / |d|^3).
// The lattice kernel unrolls its exact near pairs over these at compile time.
__host__ __device__ constexpr int near2_code(int n) {
    return n == 0 ? 3 + 5 * 2 + 25 * 2 :          // (1, 0, 0)
           n == 1 ? 2 + 5 * 3 + 25 * 2 :          // (0, 1, 0)
           n == 2 ? 2 + 5 * 2 + 25 * 3 :          // (0, 0, 1)
           n == 3 ? 3 + 5 * 3 + 25 * 2 :          // (1, 1, 0)
           n == 4 ? 3 + 5 * 1 + 25 * 2 :          // (1, -1, 0)
           n == 5 ? 3 + 5 * 2 + 25 * 3 :          // (1, 0, 1)
           n == 6 ? 3 + 5 * 2 + 25 * 1 :          // (1, 0, -1)
           n == 7 ? 2 + 5 * 3 + 25 * 3 :          // (0, 1, 1)
           n == 8 ? 2 + 5 * 3 + 25 * 1 :          // (0, 1, -1)
           n == 9 ? 3 + 5 * 3 + 25 * 3 :          // (1, 1, 1)
           n == 10 ? 3 + 5 * 3 + 25 * 1 :         // (1, 1, -1)
           n == 11 ? 3 + 5 * 1 + 25 * 3 :         // (1, -1, 1)
           n == 12 ? 3 + 5 * 1 + 25 * 1 :         // (1, -1, -1)
           n == 13 ? 4 + 5 * 2 + 25 * 2 :         // (2, 0, 0)
           n == 14 ? 2 + 5 * 4 + 25 * 2 :         // (0, 2, 0)
                     2 + 5 * 2 + 25 * 4;          // (0, 0, 2)
}
// 1/|d| and 1/|d|^3 for |d|^2 = 1, 2, 3, 4
__host__ __device__ constexpr double near2_inv_r(int r2) {
    return r2 == 1 ? 1.0 : r2 == 2 ? 0.70710678118654752440 : r2 == 3 ? 0.57735026918962576451 : 0.5;
}
__host__ __device__ constexpr double near2_inv_r3(int r2) {
    return r2 == 1 ? 1.0 : r2 == 2 ? 0.35355339059327376220 : r2 == 3 ? 0.19245008972987525484 : 0.125;
}

// Dynamic shared memory of one CTA of a kernel mode (0: FP64 all pairs,
// 1: FP64 near pairs, 2: FP32 far pairs), halo widths and staged far-table
// entries (mode 2).
size_t lattice_smem_bytes(int mode, int w_far, int w_near, int far_table_entries);

// Largest dynamic shared memory of a lattice CTA (the limit configure_lattice sets).
constexpr size_t kLatticeSmemMax = 160 * 1024;

// Fills the far-table fields of lp (n_far_max from the plan's list lengths;
// staging in shared memory when halo + tables fit in kLatticeSmemMax).
void lattice_far_table_plan(DevLattice& lp, const int* list_len);

// Raises the kernels' dynamic shared memory limit (call once per device,
// outside any stream capture); 0 on success.
int configure_lattice();

// FP64 form: one kernel on s.  FP32-bulk form: the FP64 near-pair kernel
// on s and the FP32 far-pair kernel on s_far (on s when s_far is null).
// ctas: persistent CTAs per kernel (<= 0: one per node); the node counters
// lp.counter[0..1] must be zero.
void launch_lattice(const DevTree& t, const DevPlan& p, const DevLattice& lp, int precision,
                    double G, int ctas, cudaStream_t s, cudaStream_t s_far = nullptr);

}  // namespace otfmm
