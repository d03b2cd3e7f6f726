// Launcher of the tangent (forward-mode derivative) of the solve (tangent.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace otfmm {

// Tangent arrays beside the tree's own: moments [20][cells], per-cell
// records [cells][24], expansions [23][cells] (FP64).  The moment and record
// entries of leaf cells other than the mass must be zero.
struct TanArrays {
    double* mom_d;
    double* rec_d;
    double* loc_d;
};

// phi_dot, g_dot (and phi, g when not null) of the solve for densities rho
// changing at rho_dot, FP64 dual numbers; the plan's node counters
// p.counter[0] and lp.counter[0..1] must be zero.
void launch_tangent(const DevTree& t, const TanArrays& a, const int* leaf_node, const DevPlan& p,
                    const DevLattice& lp, const int* level_first, int n_levels, const double* rho,
                    const double* rho_dot, double* phi, double* g, double* phi_dot, double* g_dot, double G,
                    int am, int self_term, int ctas, cudaStream_t s);

}  // namespace otfmm
