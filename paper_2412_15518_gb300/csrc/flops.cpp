// Algorithmic flop counts of one pair interaction of each class, taken from
// the very templates the kernels execute (pair_formula.cuh) instantiated with
// counting scalars: +, -, * and rsqrt count 1, fma counts 2, sign changes,
// constants and the exact FP32 -> FP64 widening (integer operations) count
// 0.  The split pair of the FP32-bulk form is counted with two scalars, one
// per precision.
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
inline CountT rsqrt_adj(CountT) { g_flops += 1; return CountT(); }
inline CountT operator/(CountT, CountT) { g_flops += 1; return CountT(); }
inline bool operator!=(CountT, CountT) { return true; }  // a target mass is non-zero

// The split pair: D counts into g_flops64, F into g_flops32.
static long long g_flops64 = 0, g_flops32 = 0;
struct CountD {
    CountD() {}
    CountD(double) {}
};
struct CountF {
    CountF() {}
    CountF(double) {}
};
inline CountD operator+(CountD, CountD) { g_flops64 += 1; return CountD(); }
inline CountD operator-(CountD, CountD) { g_flops64 += 1; return CountD(); }
inline CountD operator*(CountD, CountD) { g_flops64 += 1; return CountD(); }
inline CountD operator-(CountD) { return CountD(); }
inline CountD& operator+=(CountD& a, CountD) { g_flops64 += 1; return a; }
inline CountD fma_(CountD, CountD, CountD) { g_flops64 += 2; return CountD(); }
inline CountD rsqrt_(CountD) { g_flops64 += 1; return CountD(); }
inline CountF operator+(CountF, CountF) { g_flops32 += 1; return CountF(); }
inline CountF operator-(CountF, CountF) { g_flops32 += 1; return CountF(); }
inline CountF operator*(CountF, CountF) { g_flops32 += 1; return CountF(); }
inline CountF operator-(CountF) { return CountF(); }
inline CountF& operator+=(CountF& a, CountF) { g_flops32 += 1; return a; }
inline CountF fma_(CountF, CountF, CountF) { g_flops32 += 2; return CountF(); }
inline CountF rsqrt_(CountF) { g_flops32 += 1; return CountF(); }
inline CountD to_d(CountF) { return CountD(); }

}  // namespace otfmm

#include "adjoint_pair.cuh"
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

// The tangent's dual numbers: every dual operation counted as the FP64
// operations it executes (add 2, multiply 3, fma 6, reciprocal square root
// 5: the value's and the tangent's parts).
static long long g_flops_dual = 0;
struct CountDual {
    CountDual() {}
    CountDual(double) {}
};
inline CountDual operator+(CountDual, CountDual) { g_flops_dual += 2; return CountDual(); }
inline CountDual operator-(CountDual, CountDual) { g_flops_dual += 2; return CountDual(); }
inline CountDual operator*(CountDual, CountDual) { g_flops_dual += 3; return CountDual(); }
inline CountDual operator-(CountDual) { return CountDual(); }
inline CountDual& operator+=(CountDual& a, CountDual) { g_flops_dual += 2; return a; }
inline CountDual fma_(CountDual, CountDual, CountDual) { g_flops_dual += 6; return CountDual(); }
inline CountDual rsqrt_(CountDual) { g_flops_dual += 5; return CountDual(); }

template <bool FULL, bool MULTI> static double count_tangent() {
    g_flops_dual = 0;
    CountDual b2[6], b3[10], bt[4];
    Acc<CountDual> A;
    CountDual x, y, z, m;
    g_flops_dual += 12;  // R = (dX_A - dX_B) - d, dual
    m2l_pair<CountDual, FULL, MULTI, true>(x, y, z, m, b2, b3, bt, A);
    return (double)g_flops_dual;
}

void pair_flops_tangent(double out[PairClasses]) {
    // leaf-leaf pairs: the lattice kernel on the masses and on their tangents
    out[kLatticeFar] = out[kNearP2P] = 16.0;
    out[kM2P] = count_tangent<false, true>();
    out[kP2M] = count_tangent<true, false>();
    out[kMM] = count_tangent<true, true>();
}

template <bool FULL, bool MULTI> static void count_split(double& f64, double& f32) {
    g_flops64 = g_flops32 = 0;
    CountF b2[6], b3[10], bt[4];
    SplitAcc<CountD, CountF> A;
    CountD x, y, z, m;
    CountF xf, yf, zf;
    // R' = (dX_A - dX_B) - d in each precision: 2 flops per component each
    // (the FP32 copy only for a multipole source)
    g_flops64 += 6;
    if (MULTI) g_flops32 += 6;
    m2l_pair_split<CountD, CountF, FULL, MULTI, true>(x, y, z, m, xf, yf, zf, b2, b3, bt, A);
    f64 = (double)g_flops64;
    f32 = (double)g_flops32;
}

void pair_flops_split(double f64[PairClasses], double f32[PairClasses]) {
    // every leaf-leaf pair is an FP64 lattice pair: 4 fma
    f64[kLatticeFar] = f64[kNearP2P] = 8.0;
    f32[kLatticeFar] = f32[kNearP2P] = 0.0;
    count_split<false, true>(f64[kM2P], f32[kM2P]);
    count_split<true, false>(f64[kP2M], f32[kP2M]);
    count_split<true, true>(f64[kMM], f32[kMM]);
}

// The reverse of one directed pair, as the adjoint kernel runs it (with the
// correction): a pair with a leaf target in its interior source's pass
// (source adjoints and the R-gradient), a pair with an interior target whole
// in the target's pass; R formed from the offsets and the centres in cell
// units (6 flops).
// The target's partner-independent parts (reverse_target_prep) are formed
// once per interior target and not counted; a leaf target's (e0 / 2, -e0 / 6)
// are formed per pair and counted.
template <bool TGT_INTERIOR> static double count_reverse(bool multiB) {
    CountT R[3], M2B[6], M3B[10], btB[4], M3A[10], E1[3], E2[6], E3[10], ac[3], gR[3];
    CountT mB, iA, E0, oM2, oM3, oR;
    PairAdjOutT<CountT> o;
    RevTarget<CountT> tg;
    g_flops = 0;
    reverse_target_prep<TGT_INTERIOR>(E0, E2, E3, TGT_INTERIOR, iA, M3A, ac, tg);
    if (TGT_INTERIOR) g_flops = 0;
    // an interior target (pass 2) keeps the correction's mass ratio; a leaf
    // target (pass 1) has no E2, E3 or octupole
    m2l_pair_reverse<true, TGT_INTERIOR, TGT_INTERIOR>(R, mB, M2B, M3B, btB, multiB, TGT_INTERIOR, iA, M3A, E0,
                                                       E1, E2, E3, tg, true, ac, true, oM2, oM3, oR, gR, o);
    return (double)g_flops + 6.0;
}

void pair_flops_adjoint(double out[PairClasses]) {
    // leaf-leaf pairs: the lattice table transposed, 4 fma
    out[kLatticeFar] = out[kNearP2P] = 8.0;
    out[kM2P] = count_reverse<false>(true);
    out[kP2M] = count_reverse<true>(false);
    out[kMM] = count_reverse<true>(true);
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
