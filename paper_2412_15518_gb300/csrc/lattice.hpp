// Launcher of the lattice kernel (lattice.cu): leaf-leaf pairs of the leaf
// nodes of level >= 1.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "common.cuh"

namespace otfmm {

// Dynamic shared memory of one CTA for a precision and halo widths.
size_t lattice_smem_bytes(int precision, int w_far, int w_near);

// Raises the kernels' dynamic shared memory limit (call once per device,
// outside any stream capture); 0 on success.
int configure_lattice();

void launch_lattice(const DevTree& t, const DevPlan& p, const DevLattice& lp, int precision,
                    double G, cudaStream_t s);

}  // namespace otfmm
