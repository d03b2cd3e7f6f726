// Launcher of the lattice kernel (lattice.cu): leaf-leaf pairs of the leaf
// nodes of level >= 1.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "common.cuh"

namespace otfmm {

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
