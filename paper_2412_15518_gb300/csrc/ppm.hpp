// Launcher of the PPM reconstruction of the 26 directional cell values (ppm.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace otfmm {

// u: device [n_leaf][n_fields][512] cell averages of a tree whose leaves are
// all at one level (n_side = 8 * 2^level cells per axis); out: device
// [n_leaf][n_fields][26][512].
void launch_ppm(const DevTree& t, const int* leaf_node, const double* u, int n_fields, int n_side,
                double* out, cudaStream_t s);

}  // namespace otfmm
