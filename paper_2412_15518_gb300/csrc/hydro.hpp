// Launcher of the hydro right-hand side (hydro.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace otfmm {

// V: device [n_leaf][5][26][512] PPM values of the conserved fields (ppm.cu);
// u: device [n_leaf][5][512] cell averages; g: device [n_leaf][3][512]
// gravitational acceleration or null; h: cell side; dudt: device
// [n_leaf][5][512].  The tree's leaves are all at one level.
void launch_hydro_rhs(const DevTree& t, const int* leaf_node, const double* V, const double* u,
                      const double* g, double gamma, double h, double* dudt, cudaStream_t s);

}  // namespace otfmm
