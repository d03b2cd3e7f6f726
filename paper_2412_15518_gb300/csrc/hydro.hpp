// Launchers of the hydro right-hand side (hydro.cu).
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "common.cuh"

namespace otfmm {

// Doubles of the hydro workspace of a tree with n_leaf leaves: the PPM values
// of the leaves' cells (own), of the ghost cells next to their faces (ghost)
// and the fluxes of their faces (faces); returns the sum.
size_t hydro_workspace_doubles(int n_leaf, size_t* own, size_t* ghost, size_t* faces);

// u: device [n_leaf][5][512] cell averages of a 2:1-balanced tree; g: device
// [n_leaf][3][512] gravitational acceleration or null; work: device workspace
// of hydro_workspace_doubles(n_leaf) doubles; dudt: device [n_leaf][5][512].
void launch_hydro_rhs(const DevTree& t, const int* leaf_node, const double* u, const double* g, double gamma,
                      double* work, double* dudt, cudaStream_t s);

}  // namespace otfmm
