// Launchers of the GB300 FMM kernels (host side of the .cu translation units).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace otfmm {

// Upward pass: leaf masses, then exact M2M level by level (Lmax-1 .. 0).
// kinds: bit 0 the kernel for cells with interior children, bit 1 the one
// for cells with leaf children (HostTree::m2m_kinds).  precision 1 (FP32-bulk
// form): the shift products in FP32, every sum in FP64.
void launch_leaf_moments(const DevTree& t, const int* leaf_node, const double* rho,
                         cudaStream_t s);
void launch_m2m(const DevTree& t, int kinds, int first, int count, int precision, cudaStream_t s);
// The moments of nodes [first, first + count) in physical units, per node
// [20][512] (m, X, M2, M3), for ot_get_moments.
void launch_get_moments(const DevTree& t, int first, int count, double* out, cudaStream_t s);

// All cell-to-cell interactions of every level: persistent launch over the
// work items (precision 0 = FP64, 1 = FP32 bulk).
void launch_interact(const DevTree& t, const DevPlan& p, int precision, double G, int am,
                     int ctas, int warps_per_cta, cudaStream_t s);
// Sets the general kernels' shared-memory carveout (once per device, outside
// any stream capture); 0 on success.
int configure_interact();

// Downward pass for one level: L2L from the parent into the level's interior
// cells (kinds bit 0), then phi and g at the leaf cells of its children
// (bit 1) (HostTree::l2l_kinds).  precision 1 (FP32-bulk form): the shift
// arithmetic in FP32, every sum in FP64.
void launch_l2l(const DevTree& t, int kinds, int first, int count, const double* rho,
                double* phi, double* g, double G, int self_term, int precision, cudaStream_t s);

}  // namespace otfmm
