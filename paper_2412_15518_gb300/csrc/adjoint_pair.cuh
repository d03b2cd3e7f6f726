// Reverse (adjoint) of one cell-to-cell multipole interaction, FP64,
// physical units, for the hand-written adjoint of the solve.
//
// Forward pair (target A, source B, R = X_A - X_B), as in pair_formula.cuh:
//   L0_A += -G [m D0 + M2:D2 / 2 - M3:D3 / 6]
//   L1_A += -G [m D1 + (D3:M2) / 2]
//   L2_A += -G m D2,   L3_A += -G m D3
//   ac_A += -(G/6) D4 : Q,   Q = M3_B - (m_B / m_A) M3_A
// Given the adjoints E0, E1, E2, E3 (symmetric, packed) of A's expansion and
// a of its correction acceleration, this adds
//   source side: dJ/dm_B, dJ/dM2_B, dJ/dM3_B (symmetric adjoints);
//   target side: dJ/dm_A, dJ/dM3_A (through the correction's mass ratio);
//   dJ/dR (+ to X_A, - to X_B).
// With f_k = (-1)^k (2k-1)!! / r^(2k+1) and grad f_k = f_{k+1} R, every
// contraction with D^(n) is a few scalars (see pair_formula.cuh), and the
// R-gradient of each scalar is written out term by term below.
#pragma once

namespace otfmm {

struct PairAdjOut {
    double mB, M2B[6], M3B[10];
    double mA, M3A[10];
    double R[3];
};

__host__ __device__ inline void adj_zero(PairAdjOut& o) {
    o.mB = 0.0;
    o.mA = 0.0;
    for (int i = 0; i < 6; i++) o.M2B[i] = 0.0;
    for (int i = 0; i < 10; i++) {
        o.M3B[i] = 0.0;
        o.M3A[i] = 0.0;
    }
    for (int i = 0; i < 3; i++) o.R[i] = 0.0;
}

// Symmetric rank-2 (packed xx xy xz yy yz zz) times vector.
__host__ __device__ inline void sym2_vec(const double* S, const double* v, double* o) {
    o[0] = S[0] * v[0] + S[1] * v[1] + S[2] * v[2];
    o[1] = S[1] * v[0] + S[3] * v[1] + S[4] * v[2];
    o[2] = S[2] * v[0] + S[4] * v[1] + S[5] * v[2];
}

// Symmetric rank-3 (packed) contracted twice with R: q2_i = T_ijk R_j R_k.
__host__ __device__ inline void sym3_rr(const double* c, const double* R, double* q) {
    const double x = R[0], y = R[1], z = R[2];
    const double xx = x * x, yy = y * y, zz = z * z, xy2 = 2 * x * y, xz2 = 2 * x * z, yz2 = 2 * y * z;
    q[0] = c[0] * xx + c[3] * yy + c[5] * zz + c[1] * xy2 + c[2] * xz2 + c[4] * yz2;
    q[1] = c[1] * xx + c[6] * yy + c[8] * zz + c[3] * xy2 + c[4] * xz2 + c[7] * yz2;
    q[2] = c[2] * xx + c[7] * yy + c[9] * zz + c[4] * xy2 + c[5] * xz2 + c[8] * yz2;
}

// u_p = T_pik a_i R_k for a symmetric rank-3 T (packed).
__host__ __device__ inline void sym3_ab(const double* c, const double* a, const double* R, double* u) {
    // full T_pik as a function of packed indices
    const double T[3][3][3] = {
        {{c[0], c[1], c[2]}, {c[1], c[3], c[4]}, {c[2], c[4], c[5]}},
        {{c[1], c[3], c[4]}, {c[3], c[6], c[7]}, {c[4], c[7], c[8]}},
        {{c[2], c[4], c[5]}, {c[4], c[7], c[8]}, {c[5], c[8], c[9]}}};
    for (int p = 0; p < 3; p++) {
        double s = 0.0;
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) s += T[p][i][k] * a[i] * R[k];
        u[p] = s;
    }
}

__host__ __device__ inline void sym3_trace(const double* c, double* t) {
    t[0] = c[0] + c[3] + c[5];
    t[1] = c[1] + c[6] + c[8];
    t[2] = c[2] + c[7] + c[9];
}

// s4 = a . (D4 : T) and its pieces, T symmetric rank 3.
struct S4Parts {
    double q2[3], q3, t[3], Rt;
};

__host__ __device__ inline void s4_parts(const double* T, const double* R, S4Parts& s) {
    sym3_rr(T, R, s.q2);
    s.q3 = R[0] * s.q2[0] + R[1] * s.q2[1] + R[2] * s.q2[2];
    sym3_trace(T, s.t);
    s.Rt = R[0] * s.t[0] + R[1] * s.t[1] + R[2] * s.t[2];
}

// Packed symmetric rank-3 tensor (a . D4)_{jkl} for a vector a.
__host__ __device__ inline void a_dot_d4(const double* a, const double* R, double f2, double f3,
                                         double f4, double* o) {
    const int J[10] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 2};
    const int K[10] = {0, 0, 0, 1, 1, 2, 1, 1, 2, 2};
    const int Ll[10] = {0, 1, 2, 1, 2, 2, 1, 2, 2, 2};
    const double aR = a[0] * R[0] + a[1] * R[1] + a[2] * R[2];
    for (int n = 0; n < 10; n++) {
        const int j = J[n], k = K[n], l = Ll[n];
        const double djk = j == k, djl = j == l, dkl = k == l;
        o[n] = f4 * aR * R[j] * R[k] * R[l] +
               f3 * (a[j] * R[k] * R[l] + a[k] * R[j] * R[l] + a[l] * R[j] * R[k] +
                     aR * (djk * R[l] + djl * R[k] + dkl * R[j])) +
               f2 * (djk * a[l] + djl * a[k] + dkl * a[j]);
    }
}

// Reverse of one pair.  want_B: source-moment adjoints (mB always; M2B, M3B
// when the source is an interior cell).  want_A: the target-side mass-ratio
// adjoints (interior targets only).  want_R: dJ/dR.
__host__ __device__ inline void m2l_pair_reverse(
    const double* Rv, double G, int am,
    double mB, const double* M2B, const double* M3B, bool multiB,   // source moments
    double mA, const double* M3A, bool multiA,                      // target moments (ratio)
    double E0, const double* E1, const double* E2, const double* E3, const double* ac,
    bool want_B, bool want_A, bool want_R, PairAdjOut& out) {
    const double x = Rv[0], y = Rv[1], z = Rv[2];
    const double r2 = x * x + y * y + z * z;
    const double r = sqrt(r2);
    const double f0 = 1.0 / r;
    const double ri2 = f0 * f0;
    const double f1 = -f0 * ri2;
    const double f2 = -3.0 * f1 * ri2;
    const double f3 = -5.0 * f2 * ri2;
    const double f4 = -7.0 * f3 * ri2;
    const double f5 = -9.0 * f4 * ri2;
    const double R[3] = {x, y, z};
    // the target's M3 enters only through the correction's mass-ratio term,
    // which is taken as zero (and has no derivative) for a target of zero mass
    const bool useA = am && multiA && mA != 0.0;
    const double ratio = useA ? mB / mA : 0.0;

    // contractions of the adjoints with R
    const double E1R = E1[0] * x + E1[1] * y + E1[2] * z;
    double E2R[3];
    sym2_vec(E2, R, E2R);
    const double RE2R = E2R[0] * x + E2R[1] * y + E2R[2] * z;
    const double trE2 = E2[0] + E2[3] + E2[5];
    S4Parts e3;
    s4_parts(E3, R, e3);
    const double aR = am ? ac[0] * x + ac[1] * y + ac[2] * z : 0.0;
    S4Parts qa;  // target M3 (ratio part)
    if (useA) s4_parts(M3A, R, qa);

    if (want_B) {
        // dJ/dm_B
        double v = E0 * f0 + f1 * E1R + f2 * RE2R + f1 * trE2 + f3 * e3.q3 + 3.0 * f2 * e3.Rt;
        out.mB += -G * v;
        if (useA) {
            const double s4a = f4 * aR * qa.q3 +
                               3.0 * f3 * (ac[0] * qa.q2[0] + ac[1] * qa.q2[1] + ac[2] * qa.q2[2] + aR * qa.Rt) +
                               3.0 * f2 * (ac[0] * qa.t[0] + ac[1] * qa.t[1] + ac[2] * qa.t[2]);
            out.mB += (G / 6.0) / mA * s4a;
        }
        if (multiB) {
            // dJ/dM2_B = -G [E0 D2 / 2 + (E1 . D3) / 2]
            const int I2[6] = {0, 0, 0, 1, 1, 2}, J2[6] = {0, 1, 2, 1, 2, 2};
            for (int n = 0; n < 6; n++) {
                const int j = I2[n], k = J2[n];
                const double djk = j == k;
                const double d2 = f2 * R[j] * R[k] + f1 * djk;
                const double e1d3 = f3 * E1R * R[j] * R[k] + f2 * (E1[j] * R[k] + E1[k] * R[j] + djk * E1R);
                out.M2B[n] += -G * 0.5 * (E0 * d2 + e1d3);
            }
            // dJ/dM3_B = -G (-E0 D3 / 6) - (G/6) a . D4
            const int J[10] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 2};
            const int K[10] = {0, 0, 0, 1, 1, 2, 1, 1, 2, 2};
            const int Ll[10] = {0, 1, 2, 1, 2, 2, 1, 2, 2, 2};
            double ad4[10];
            if (am) a_dot_d4(ac, R, f2, f3, f4, ad4);
            for (int n = 0; n < 10; n++) {
                const int j = J[n], k = K[n], l = Ll[n];
                const double d3 = f3 * R[j] * R[k] * R[l] +
                                  f2 * ((j == k) * R[l] + (j == l) * R[k] + (k == l) * R[j]);
                out.M3B[n] += -G * (-(1.0 / 6.0)) * E0 * d3;
                if (am) out.M3B[n] += -(G / 6.0) * ad4[n];
            }
        }
    }
    if (want_A && useA) {
        double ad4[10];
        a_dot_d4(ac, R, f2, f3, f4, ad4);
        for (int n = 0; n < 10; n++) out.M3A[n] += (G / 6.0) * ratio * ad4[n];
        const double s4a = f4 * aR * qa.q3 +
                           3.0 * f3 * (ac[0] * qa.q2[0] + ac[1] * qa.q2[1] + ac[2] * qa.q2[2] + aR * qa.Rt) +
                           3.0 * f2 * (ac[0] * qa.t[0] + ac[1] * qa.t[1] + ac[2] * qa.t[2]);
        out.mA += -(G / 6.0) * s4a * (mB / (mA * mA));
    }
    if (want_R) {
        double g[3] = {0.0, 0.0, 0.0};
        // T1 = m E0 D0 ; T4 = m E1 . D1 ; T6 = m E2 : D2 ; T7 = m E3 : D3
        for (int p = 0; p < 3; p++) {
            g[p] += mB * E0 * f1 * R[p];
            g[p] += mB * (f1 * E1[p] + f2 * E1R * R[p]);
            g[p] += mB * (f3 * RE2R * R[p] + 2.0 * f2 * E2R[p] + f2 * trE2 * R[p]);
            g[p] += mB * (f4 * e3.q3 * R[p] + 3.0 * f3 * e3.q2[p] + 3.0 * f3 * e3.Rt * R[p] +
                          3.0 * f2 * e3.t[p]);
        }
        if (multiB) {
            // T2 = E0 M2 : D2 / 2
            double MR[3];
            sym2_vec(M2B, R, MR);
            const double xMx = MR[0] * x + MR[1] * y + MR[2] * z;
            const double trM = M2B[0] + M2B[3] + M2B[5];
            double ME1[3];
            sym2_vec(M2B, E1, ME1);
            const double E1MR = E1[0] * MR[0] + E1[1] * MR[1] + E1[2] * MR[2];
            S4Parts m3;
            s4_parts(M3B, R, m3);
            for (int p = 0; p < 3; p++) {
                g[p] += 0.5 * E0 * (f3 * xMx * R[p] + 2.0 * f2 * MR[p] + f2 * trM * R[p]);
                // T3 = -E0 M3 : D3 / 6
                g[p] += -(1.0 / 6.0) * E0 *
                        (f4 * m3.q3 * R[p] + 3.0 * f3 * m3.q2[p] + 3.0 * f3 * m3.Rt * R[p] + 3.0 * f2 * m3.t[p]);
                // T5 = E1 . (D3 : M2) / 2
                g[p] += 0.5 * (f4 * E1R * xMx * R[p] + f3 * (E1[p] * xMx + 2.0 * E1R * MR[p]) +
                               f3 * (2.0 * E1MR + E1R * trM) * R[p] + f2 * (2.0 * ME1[p] + E1[p] * trM));
            }
        }
        for (int p = 0; p < 3; p++) out.R[p] += -G * g[p];
        if (am) {
            // T8 = a . (D4 : Q), Q = M3_B - ratio M3_A
            double Q[10];
            for (int n = 0; n < 10; n++)
                Q[n] = (multiB ? M3B[n] : 0.0) - (useA ? ratio * M3A[n] : 0.0);
            S4Parts q;
            s4_parts(Q, R, q);
            double u[3];
            sym3_ab(Q, ac, R, u);
            const double aq2 = ac[0] * q.q2[0] + ac[1] * q.q2[1] + ac[2] * q.q2[2];
            const double at = ac[0] * q.t[0] + ac[1] * q.t[1] + ac[2] * q.t[2];
            for (int p = 0; p < 3; p++) {
                const double v = R[p] * (f5 * aR * q.q3 + 3.0 * f4 * aq2 + 3.0 * f4 * aR * q.Rt + 3.0 * f3 * at) +
                                 ac[p] * (f4 * q.q3 + 3.0 * f3 * q.Rt) + 3.0 * f4 * aR * q.q2[p] +
                                 6.0 * f3 * u[p] + 3.0 * f3 * aR * q.t[p];
                out.R[p] += -(G / 6.0) * v;
            }
        }
    }
}

}  // namespace otfmm
