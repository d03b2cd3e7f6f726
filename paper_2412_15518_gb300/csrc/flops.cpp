// Algorithmic flop counts of one pair interaction of each class, taken from
// the very template the kernels execute (pair_formula.cuh) instantiated with
// a counting scalar: +, -, * and rsqrt count 1, fma counts 2, sign changes
// and constants count 0.
#include <cuda_runtime.h>

#include <cmath>

#include "tree_host.hpp"

namespace otfmm {

struct CountT {
    CountT() {}
    CountT(double) {}
};

static long long g_flops = 0;

inline CountT operator+(CountT, CountT) { g_flops += 1; return CountT(); }
inline CountT operator-(CountT, CountT) { g_flops += 1; return CountT(); }
inline CountT operator*(CountT, CountT) { g_flops += 1; return CountT(); }
inline CountT operator-(CountT) { return CountT(); }
inline CountT& operator+=(CountT& a, CountT) { g_flops += 1; return a; }
inline CountT fma_(CountT, CountT, CountT) { g_flops += 2; return CountT(); }
inline CountT rsqrt_(CountT) { g_flops += 1; return CountT(); }

}  // namespace otfmm

#include "pair_formula.cuh"

namespace otfmm {

template <bool FULL, bool MULTI, bool AM> static double count_pair() {
    g_flops = 0;
    CountT b2[6], b3[10], bt[4];
    Acc<CountT> A;
    CountT x, y, z, m;
    // R' = d + (dX_A - dX_B): 2 flops per component
    g_flops += 6;
    m2l_pair<CountT, FULL, MULTI, AM>(x, y, z, m, b2, b3, bt, A);
    return (double)g_flops;
}

void pair_flops(double out[PairClasses][2]) {
    // lattice pairs (far or near, two leaf cells): 4 fma
    out[kLatticeFar][0] = out[kLatticeFar][1] = 8.0;
    out[kNearP2P][0] = out[kNearP2P][1] = 8.0;
    out[kM2P][1] = count_pair<false, true, true>();
    out[kM2P][0] = count_pair<false, true, false>();
    out[kP2M][1] = count_pair<true, false, true>();
    out[kP2M][0] = count_pair<true, false, false>();
    out[kMM][1] = count_pair<true, true, true>();
    out[kMM][0] = count_pair<true, true, false>();
}

}  // namespace otfmm
