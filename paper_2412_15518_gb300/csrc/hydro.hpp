// Launchers of the hydro right-hand side (hydro.cu).
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "common.cuh"

namespace otfmm {

// Doubles of the hydro workspace of a tree with n_leaf leaves: the PPM values
// of the leaves' cells and their primitive variables (own), the PPM values
// of the ghost cells next to their faces (ghost) and the fluxes of their
// faces (faces); returns the sum.
size_t hydro_workspace_doubles(int n_leaf, size_t* own, size_t* ghost, size_t* faces);

// u: device [n_leaf][5][512] cell averages of a 2:1-balanced tree; g: device
// [n_leaf][3][512] gravitational acceleration or null; work: device workspace
// of hydro_workspace_doubles(n_leaf) doubles; dudt: device [n_leaf][5][512].
void launch_hydro_rhs(const DevTree& t, const int* leaf_node, const double* u, const double* g, double gamma,
                      double* work, double* dudt, cudaStream_t s);

// rho[leaf][c] = U[leaf][0][c] (the density of a state, for its gravity solve).
void launch_stage_density(const double* U, double* rho, int n_leaf, cudaStream_t s);

// One combination of the third-order SSP Runge-Kutta scheme: stage 1
// out = U0 + dt L, stage 2 out = 3/4 U0 + 1/4 (Uc + dt L), stage 3
// out = 1/3 U0 + 2/3 (Uc + dt L); out may be Uc.
void launch_rk3_combine(const double* U0, const double* Uc, const double* L, double dt, int stage, double* out,
                        int n_leaf, cudaStream_t s);

}  // namespace otfmm
