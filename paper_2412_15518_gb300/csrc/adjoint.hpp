// Launchers of the adjoint kernels (adjoint.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace otfmm {

void launch_adj_seed(const DevTree& t, const int* leaf_node, const double* w1, const double* w2,
                     double* locbar, cudaStream_t s);
void launch_l2l_reverse(const DevTree& t, int first, int count, double* locbar, double* mombar,
                        cudaStream_t s);
void launch_m2l_reverse(const DevTree& t, const DevPlan& p, const double* locbar, double* mombar,
                        double G, int am, int ctas, cudaStream_t s);
void launch_m2m_reverse(const DevTree& t, int first, int count, double* mombar, cudaStream_t s);
void launch_rho_bar(const DevTree& t, const int* leaf_node, const double* mombar, const double* w1,
                    double* drho, double G, int self_term, cudaStream_t s);

}  // namespace otfmm
