// Launcher of the lattice kernel (lattice.cu): leaf-leaf pairs of the leaf
// nodes of level >= 1.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "common.cuh"

namespace otfmm {

// Dynamic shared memory of one CTA of a kernel mode (0: FP64 all pairs,
// 1: FP64 near pairs, 2: FP32 far pairs) and halo widths.
size_t lattice_smem_bytes(int mode, int w_far, int w_near);

// Raises the kernels' dynamic shared memory limit (call once per device,
// outside any stream capture); 0 on success.
int configure_lattice();

// FP64 form: one kernel on s.  FP32-bulk form: the FP64 near-pair kernel
// on s and the FP32 far-pair kernel on s_far (on s when s_far is null).
void launch_lattice(const DevTree& t, const DevPlan& p, const DevLattice& lp, int precision,
                    double G, cudaStream_t s, cudaStream_t s_far = nullptr);

}  // namespace otfmm
