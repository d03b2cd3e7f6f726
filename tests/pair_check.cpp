// Evaluates the GPU library's own pair formulas on the host -- the forward
// cell-to-cell interaction (pair_formula.cuh: m2l_pair, the Kronecker parts
// from the traces, the correction's target term) and its reverse
// (adjoint_pair.cuh: m2l_pair_reverse) -- for pairs read from stdin, in FP64
// and physical units (cell side 1), so that a test can compare them with
// the oracle's unpacked formulation.
//
// Input, one pair per line: am G  XA[3] XB[3]  mA M3A[10]  mB M2B[6] M3B[10]
//   E0 E1[3] E2[6] E3[10] a[3]       (symmetric tensors packed: xx xy xz yy
//   yz zz; xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz)
// Output, one line per pair: the expansion at A due to B, L0 L1[3] L2[6]
// L3[10] ac[3]; then the reverse given the adjoints (E, a): dJ/dmB,
// dJ/dM2B[6], dJ/dM3B[10], dJ/dmA, dJ/dM3A[10], dJ/dR[3] (R = XA - XB);
// then the same expansion from the FP32-bulk form's split pair
// (m2l_pair_split) twice: with both scalars double (the split's algebra),
// and with the FP32 part in float (R, M2, M3 rounded to float as the FP32
// records hold them); then the reverse again in cell units of side 0.37 (as
// the adjoint kernel runs it), in physical units; then the reverse for a
// leaf target (no E2, E3 or octupole): dJ/dmB, dJ/dM2B[6], dJ/dM3B[10],
// dJ/dR[3].
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "../paper_2412_15518_gb300/csrc/pair_formula.cuh"
#include "../paper_2412_15518_gb300/csrc/adjoint_pair.cuh"

using namespace otfmm;

static bool rd(double* v, int n) {
    for (int i = 0; i < n; i++)
        if (std::scanf("%lf", v + i) != 1) return false;
    return true;
}

static void trace3(const double* c, double* t) {
    t[0] = c[0] + c[3] + c[5];
    t[1] = c[1] + c[6] + c[8];
    t[2] = c[2] + c[7] + c[9];
}

// The split pair's expansion at A due to B, as the FP32-bulk kernel
// assembles it (F partial sums flushed into the D sums, Kronecker parts,
// correction's target term), physical units.
template <class F>
static void split_out(int am, double G, const double* R, double mA, const double* M3A, double mB,
                      const double* M2B, const double* M3B, const double* bt) {
    SplitAcc<double, F> A;
    split_zero(A);
    F b2[6], b3[10], tf[4];
    for (int r = 0; r < 6; r++) b2[r] = (F)M2B[r];
    for (int r = 0; r < 10; r++) b3[r] = (F)M3B[r];
    for (int r = 0; r < 4; r++) tf[r] = (F)bt[r];
    const F xf = (F)R[0], yf = (F)R[1], zf = (F)R[2];
    if (am)
        m2l_pair_split<double, F, true, true, true>(R[0], R[1], R[2], mB, xf, yf, zf, b2, b3, tf, A);
    else
        m2l_pair_split<double, F, true, true, false>(R[0], R[1], R[2], mB, xf, yf, zf, b2, b3, tf, A);
    flush_split(A);
    finish_split(A);
    double P[3] = {0.0, 0.0, 0.0};
    if (am && mA != 0.0) {
        double a3[10], ta[3];
        for (int r = 0; r < 10; r++) a3[r] = M3A[r] / mA;
        trace3(a3, ta);
        correction_target_split(A, a3, ta, P);
    }
    std::printf(" %.17g", -G * A.L0);
    for (double v : A.L1) std::printf(" %.17g", -G * v);
    for (double v : A.L2) std::printf(" %.17g", -G * v);
    for (double v : A.L3) std::printf(" %.17g", -G * v);
    for (int i = 0; i < 3; i++) std::printf(" %.17g", am ? -(G / 6.0) * (A.S[i] - P[i]) : 0.0);
}

// The reverse pair with an interior target (both roles and the R-gradient)
// in cell units of side h, its outputs printed in physical units: dJ/dmB,
// dJ/dM2B, dJ/dM3B, dJ/dmA, dJ/dM3A, dJ/dR.  The target's quartic sum comes
// from reverse_target_quartic, or (from_forward, as the adjoint kernel takes
// it) from the forward pair's own sum Acc::A4 times kAccCor.
static void reverse_out(int am, double G, double h, const double* R, double mA, const double* M3A,
                        double mB, const double* M2B, const double* M3B, double E0, const double* E1,
                        const double* E2, const double* E3, const double* a, bool from_forward) {
    const double hi = 1.0 / h;
    double Rc[3], M2c[6], M3Bc[10], M3Ac[10], e1[3], e2[6], e3[10], al[3];
    for (int r = 0; r < 3; r++) {
        Rc[r] = R[r] * hi;
        e1[r] = -G * hi * hi * E1[r];
        al[r] = (-G / 6.0) * hi * hi * a[r];
    }
    for (int r = 0; r < 6; r++) {
        M2c[r] = M2B[r] * hi * hi;
        e2[r] = -G * hi * hi * hi * E2[r];
    }
    for (int r = 0; r < 10; r++) {
        M3Bc[r] = M3B[r] * hi * hi * hi;
        M3Ac[r] = M3A[r] * hi * hi * hi;
        e3[r] = -G * hi * hi * hi * hi * E3[r];
    }
    const bool useA = am && mA != 0.0;
    const double iA = useA ? 1.0 / mA : 0.0;
    PairAdjOut o;
    adj_zero(o);
    double gR[3] = {0.0, 0.0, 0.0}, btB[4];
    trace3(M3Bc, btB);
    btB[3] = M2c[0] + M2c[3] + M2c[5];
    RevTarget<double> tg;
    reverse_target_prep<true>(-G * hi * E0, e2, e3, useA, iA, M3Ac, al, tg);
    m2l_pair_reverse<true, true, true>(Rc, mB, M2c, M3Bc, btB, true, useA, iA, M3Ac, -G * hi * E0, e1, e2, e3,
                                       tg, am != 0, al, true, hi * hi, hi * hi * hi, hi, gR, o);
    // the quartic sum of the target's pairs (here one)
    if (from_forward) {
        Acc<double> F;
        acc_zero(F);
        double btc[4];
        trace3(M3Bc, btc);
        btc[3] = M2c[0] + M2c[3] + M2c[5];
        m2l_pair<double, true, true, true>(Rc[0], Rc[1], Rc[2], mB, M2c, M3Bc, btc, F);
        for (int r = 0; r < 15; r++) o.A4[r] = kAccCor * F.A4[r];
    } else {
        reverse_target_quartic(Rc, mB, o);
    }
    if (useA) reverse_target_finish(o, al, -hi * hi * hi / mA);
    std::printf(" %.17g", o.mB);
    for (double v : o.M2B) std::printf(" %.17g", v);
    for (double v : o.M3B) std::printf(" %.17g", v);
    std::printf(" %.17g", o.mA);
    for (double v : o.M3A) std::printf(" %.17g", v);
    for (double v : gR) std::printf(" %.17g", v);
}

int main() {
    int am;
    double G;
    while (std::scanf("%d %lf", &am, &G) == 2) {
        double XA[3], XB[3], mA, M3A[10], mB, M2B[6], M3B[10], E0, E1[3], E2[6], E3[10], a[3];
        if (!(rd(XA, 3) && rd(XB, 3) && rd(&mA, 1) && rd(M3A, 10) && rd(&mB, 1) && rd(M2B, 6) &&
              rd(M3B, 10) && rd(&E0, 1) && rd(E1, 3) && rd(E2, 6) && rd(E3, 10) && rd(a, 3)))
            return 1;
        const double R[3] = {XA[0] - XB[0], XA[1] - XB[1], XA[2] - XB[2]};
        // forward, as the general kernel assembles it for an interior target
        Acc<double> A;
        acc_zero(A);
        double bt[4];
        trace3(M3B, bt);
        bt[3] = M2B[0] + M2B[3] + M2B[5];
        if (am)
            m2l_pair<double, true, true, true>(R[0], R[1], R[2], mB, M2B, M3B, bt, A);
        else
            m2l_pair<double, true, true, false>(R[0], R[1], R[2], mB, M2B, M3B, bt, A);
        finish_acc(A);
        double P[3] = {0.0, 0.0, 0.0};
        if (am && mA != 0.0) {
            double a3[10], ta[3];
            for (int r = 0; r < 10; r++) a3[r] = M3A[r] / mA;
            trace3(a3, ta);
            correction_target(A, a3, ta, P);
        }
        // the sums are held without their radial constants
        std::printf("%.17g", -G * A.L0);
        for (double v : A.L1) std::printf(" %.17g", -G * v);
        for (double v : A.L2) std::printf(" %.17g", -G * kAccL2 * v);
        for (double v : A.L3) std::printf(" %.17g", -G * kAccL3 * v);
        for (int i = 0; i < 3; i++)
            std::printf(" %.17g", am ? -(G / 6.0) * kAccCor * (A.S[i] - P[i]) : 0.0);
        // reverse of the same pair, both roles and the R-gradient, as the
        // adjoint kernel's pass 2 runs it (an interior target): physical
        // units are cell units with h = 1, the adjoints pre-scaled by -G and
        // -G/6
        reverse_out(am, G, 1.0, R, mA, M3A, mB, M2B, M3B, E0, E1, E2, E3, a, false);
        split_out<double>(am, G, R, mA, M3A, mB, M2B, M3B, bt);
        split_out<float>(am, G, R, mA, M3A, mB, M2B, M3B, bt);
        // the same in the kernel's cell units (side h = 0.37): R, M2, M3
        // divided by h, h^2, h^3, the adjoints scaled by h^-(n+1) and h^-2,
        // the moment and R adjoints brought back by h^-2, h^-3, h^-1, and the
        // quartic sum from the forward pair, as the kernel takes it
        reverse_out(am, G, 0.37, R, mA, M3A, mB, M2B, M3B, E0, E1, E2, E3, a, true);
        // a leaf target (pass 1): no E2, E3, octupole or mass ratio
        {
            PairAdjOut o;
            adj_zero(o);
            double gR[3] = {0.0, 0.0, 0.0}, e1[3], al[3], btB[4];
            for (int r = 0; r < 3; r++) {
                e1[r] = -G * E1[r];
                al[r] = (-G / 6.0) * a[r];
            }
            trace3(M3B, btB);
            btB[3] = M2B[0] + M2B[3] + M2B[5];
            RevTarget<double> tg;
            reverse_target_prep<false>(-G * E0, (const double*)nullptr, (const double*)nullptr, false, 0.0,
                                       (const double*)nullptr, al, tg);
            m2l_pair_reverse<true, false, false, double>(R, mB, M2B, M3B, btB, true, false, 0.0, M3A, -G * E0, e1,
                                                         nullptr, nullptr, tg, am != 0, al, true, 1.0, 1.0, 1.0,
                                                         gR, o);
            std::printf(" %.17g", o.mB);
            for (double v : o.M2B) std::printf(" %.17g", v);
            for (double v : o.M3B) std::printf(" %.17g", v);
            for (double v : gR) std::printf(" %.17g", v);
        }
        std::printf("\n");
    }
    return 0;
}
