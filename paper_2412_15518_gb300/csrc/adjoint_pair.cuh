// Reverse (adjoint) of one cell-to-cell multipole interaction, FP64,
// physical units, for the hand-written adjoint of the solve.
//
// Forward pair (target A, source B, R = X_A - X_B), as in pair_formula.cuh:
//   L0_A += -G [m D0 + M2:D2 / 2 - M3:D3 / 6]
//   L1_A += -G [m D1 + (D3:M2) / 2]
//   L2_A += -G m D2,   L3_A += -G m D3
//   ac_A += -(G/6) D4 : Q,   Q = M3_B - (m_B / m_A) M3_A
// Given the adjoints E0, E1, E2, E3 (symmetric, packed; the adjoint pairs
// with the full tensor, so an off-diagonal packed entry stands for both of
// its positions) of A's expansion and a of its correction acceleration, this
// adds
//   source side (SRC): dJ/dm_B, dJ/dM2_B, dJ/dM3_B (symmetric adjoints);
//   target side (TGT): dJ/dm_A, dJ/dM3_A (through the correction's mass ratio);
//   dJ/dR (+ to X_A, - to X_B) when want_R.
// With f_k = (-1)^k (2k-1)!! / r^(2k+1) and grad f_k = f_{k+1} R, every
// contraction with D^(n) is a few scalars (see pair_formula.cuh):
//   D2_jk = f2 R_j R_k + f1 d_jk
//   D3_jkl = f3 R_j R_k R_l + f2 (d_jk R_l + d_jl R_k + d_kl R_j)
//   (a.D4)_jkl = f4 aR RRR + f3 (aRR + aR dR) + f2 da      (packed below)
// and the R-gradient of each scalar is written out term by term.  Every
// tensor is handled through shared monomials of R (RR, RRR) with all loops
// unrolled, so nothing is indexed at run time.
#pragma once

namespace otfmm {

template <class T> struct PairAdjOutT {
    T mB, M2B[6], M3B[10];
    T mA, M3A[10];
    T R[3];
    T A4[15];  // target side: sum over partners of m_B f4 R^4 (reverse_target_finish)
};
using PairAdjOut = PairAdjOutT<double>;

template <class T> __host__ __device__ __forceinline__ void adj_zero(PairAdjOutT<T>& o) {
    o.mB = 0.0;
    o.mA = 0.0;
#pragma unroll
    for (int i = 0; i < 6; i++) o.M2B[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 10; i++) {
        o.M3B[i] = 0.0;
        o.M3A[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < 3; i++) o.R[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 15; i++) o.A4[i] = 0.0;
}

// Symmetric rank-2 (packed xx xy xz yy yz zz) times vector.
template <class T>
__host__ __device__ __forceinline__ void sym2_vec(const T* S, const T* v, T* o) {
    o[0] = S[0] * v[0] + S[1] * v[1] + S[2] * v[2];
    o[1] = S[1] * v[0] + S[3] * v[1] + S[4] * v[2];
    o[2] = S[2] * v[0] + S[4] * v[1] + S[5] * v[2];
}

// o_i = T_ijk P_jk for a packed symmetric rank-3 T (xxx xxy xxz xyy xyz xzz
// yyy yyz yzz zzz) and a symmetric P given as (P_xx, P_yy, P_zz, 2 P_xy,
// 2 P_xz, 2 P_yz): with P = R R this is T : R R.
template <class T>
__host__ __device__ __forceinline__ void sym3_contract(const T* c, T pxx, T pyy,
                                                       T pzz, T pxy2, T pxz2,
                                                       T pyz2, T* o) {
    o[0] = c[0] * pxx + c[3] * pyy + c[5] * pzz + c[1] * pxy2 + c[2] * pxz2 + c[4] * pyz2;
    o[1] = c[1] * pxx + c[6] * pyy + c[8] * pzz + c[3] * pxy2 + c[4] * pxz2 + c[7] * pyz2;
    o[2] = c[2] * pxx + c[7] * pyy + c[9] * pzz + c[4] * pxy2 + c[5] * pxz2 + c[8] * pyz2;
}

// Symmetric rank-3 (packed) contracted twice with R: q2_i = T_ijk R_j R_k.
template <class T>
__host__ __device__ __forceinline__ void sym3_rr(const T* c, const T* R, T* q) {
    const T x = R[0], y = R[1], z = R[2];
    sym3_contract(c, x * x, y * y, z * z, 2 * x * y, 2 * x * z, 2 * y * z, q);
}

// (T d)_n = T_uvl d_l for a packed symmetric rank-3 T: a packed rank-2 result.
template <class T>
__host__ __device__ __forceinline__ void sym3_vec(const T* c, const T* d, T* o) {
    o[0] = c[0] * d[0] + c[1] * d[1] + c[2] * d[2];
    o[1] = c[1] * d[0] + c[3] * d[1] + c[4] * d[2];
    o[2] = c[2] * d[0] + c[4] * d[1] + c[5] * d[2];
    o[3] = c[3] * d[0] + c[6] * d[1] + c[7] * d[2];
    o[4] = c[4] * d[0] + c[7] * d[1] + c[8] * d[2];
    o[5] = c[5] * d[0] + c[8] * d[1] + c[9] * d[2];
}

template <class T>
__host__ __device__ __forceinline__ void sym3_trace(const T* c, T* t) {
    t[0] = c[0] + c[3] + c[5];
    t[1] = c[1] + c[6] + c[8];
    t[2] = c[2] + c[7] + c[9];
}

// The pieces of a . (D4 : T) for a symmetric rank-3 T: q2 = T:RR, q3 = R.q2,
// t_i = T_ijj, Rt = R.t.
template <class T> struct S4Parts {
    T q2[3], q3, t[3], Rt;
};

// Shared monomials of R.
template <class T> struct RMono {
    T x, y, z;
    T xx, xy, xz, yy, yz, zz;   // R R
    T xy2, xz2, yz2;            // doubled cross products
    T rrr[10];                  // R R R, packed
};

template <class T>
__host__ __device__ __forceinline__ void r_mono(T x, T y, T z, RMono<T>& m) {
    m.x = x; m.y = y; m.z = z;
    m.xx = x * x; m.xy = x * y; m.xz = x * z; m.yy = y * y; m.yz = y * z; m.zz = z * z;
    m.xy2 = m.xy + m.xy; m.xz2 = m.xz + m.xz; m.yz2 = m.yz + m.yz;
    m.rrr[0] = m.xx * x; m.rrr[1] = m.xx * y; m.rrr[2] = m.xx * z; m.rrr[3] = m.yy * x;
    m.rrr[4] = m.xy * z; m.rrr[5] = m.zz * x; m.rrr[6] = m.yy * y; m.rrr[7] = m.yy * z;
    m.rrr[8] = m.zz * y; m.rrr[9] = m.zz * z;
}

template <class T>
__host__ __device__ __forceinline__ void s4_parts(const T* Tm, const RMono<T>& m, S4Parts<T>& s) {
    sym3_contract(Tm, m.xx, m.yy, m.zz, m.xy2, m.xz2, m.yz2, s.q2);
    s.q3 = m.x * s.q2[0] + m.y * s.q2[1] + m.z * s.q2[2];
    sym3_trace(Tm, s.t);
    s.Rt = m.x * s.t[0] + m.y * s.t[1] + m.z * s.t[2];
}

// o_n += c4 (RRR)_n + c3 (aRR)_n + c3r (dR)_n + c2 (da)_n over the packed
// rank-3 index n, where (aRR)_jkl = a_j R_k R_l + a_k R_j R_l + a_l R_j R_k,
// (dR)_jkl = d_jk R_l + d_jl R_k + d_kl R_j and (da) likewise with a.  With
// c4 = f4 aR, c3 = f3, c3r = f3 aR, c2 = f2 this adds a . D4; with c3 = c2 =
// 0, c4 = f3, c3r = f2 it adds D3.
template <class T>
__host__ __device__ __forceinline__ void add_rank3(T* o, const RMono<T>& m, const T* a,
                                                   T c4, T c3, T c3r, T c2) {
    const T ax = a[0], ay = a[1], az = a[2];
    const T x = m.x, y = m.y, z = m.z;
    o[0] += c4 * m.rrr[0] + c3 * (3.0 * ax * m.xx) + c3r * (3.0 * x) + c2 * (3.0 * ax);
    o[1] += c4 * m.rrr[1] + c3 * (2.0 * ax * m.xy + ay * m.xx) + c3r * y + c2 * ay;
    o[2] += c4 * m.rrr[2] + c3 * (2.0 * ax * m.xz + az * m.xx) + c3r * z + c2 * az;
    o[3] += c4 * m.rrr[3] + c3 * (ax * m.yy + 2.0 * ay * m.xy) + c3r * x + c2 * ax;
    o[4] += c4 * m.rrr[4] + c3 * (ax * m.yz + ay * m.xz + az * m.xy);
    o[5] += c4 * m.rrr[5] + c3 * (ax * m.zz + 2.0 * az * m.xz) + c3r * x + c2 * ax;
    o[6] += c4 * m.rrr[6] + c3 * (3.0 * ay * m.yy) + c3r * (3.0 * y) + c2 * (3.0 * ay);
    o[7] += c4 * m.rrr[7] + c3 * (2.0 * ay * m.yz + az * m.yy) + c3r * z + c2 * az;
    o[8] += c4 * m.rrr[8] + c3 * (ay * m.zz + 2.0 * az * m.yz) + c3r * y + c2 * ay;
    o[9] += c4 * m.rrr[9] + c3 * (3.0 * az * m.zz) + c3r * (3.0 * z) + c2 * (3.0 * az);
}

#ifdef __CUDA_ARCH__
__device__ __forceinline__ double rsqrt_adj(double a) { return rsqrt(a); }
#else
inline double rsqrt_adj(double a) { return 1.0 / sqrt(a); }
#endif

// Reverse of one pair, added into out.  SRC: source-moment adjoints (mB
// always; M2B, M3B when the source is an interior cell).  TGT: the
// target-side mass-ratio adjoints (interior targets only).  want_R: dJ/dR,
// added to gR times sR (+1 for the target's centre of mass, -1 for the
// source's).
template <bool SRC, bool TGT, class T>
__host__ __device__ __forceinline__ void m2l_pair_reverse(
    const T* Rv, T G, int am,
    T mB, const T* M2B, const T* M3B, bool multiB,   // source moments
    T mA, const T* M3A, bool multiA,                      // target moments (ratio)
    T E0, const T* E1, const T* E2, const T* E3, const T* ac,
    bool want_R, T sR, T* gR, PairAdjOutT<T>& out) {
    RMono<T> m;
    r_mono(Rv[0], Rv[1], Rv[2], m);
    const T x = m.x, y = m.y, z = m.z;
    const T R[3] = {x, y, z};
    const T f0 = rsqrt_adj(m.xx + m.yy + m.zz);
    const T ri2 = f0 * f0;
    const T f1 = -f0 * ri2;
    const T f2 = -3.0 * f1 * ri2;
    const T f3 = -5.0 * f2 * ri2;
    const T f4 = -7.0 * f3 * ri2;
    const T f5 = -9.0 * f4 * ri2;
    const T k6 = G / 6.0;
    // the target's M3 enters only through the correction's mass-ratio term,
    // which is taken as zero (and has no derivative) for a target of zero mass
    const bool useA = am && multiA && mA != 0.0;
    const T iA = useA ? 1.0 / mA : 0.0;
    const T ratio = mB * iA;
    const T zero3[3] = {0.0, 0.0, 0.0};
    const T* a = am ? ac : zero3;
    const T aR = a[0] * x + a[1] * y + a[2] * z;

    // contractions of the adjoints with R
    const T E1R = E1[0] * x + E1[1] * y + E1[2] * z;
    T E2R[3];
    sym2_vec(E2, R, E2R);
    const T RE2R = E2R[0] * x + E2R[1] * y + E2R[2] * z;
    const T trE2 = E2[0] + E2[3] + E2[5];
    S4Parts<T> e3;
    s4_parts(E3, m, e3);
    // s4a = a . (D4 : M3_A) (the ratio part of the correction)
    T s4a = 0.0;
    S4Parts<T> qa;
    if (useA) {
        s4_parts(M3A, m, qa);
        s4a = f4 * aR * qa.q3 + 3.0 * f3 * (a[0] * qa.q2[0] + a[1] * qa.q2[1] + a[2] * qa.q2[2] + aR * qa.Rt) +
              3.0 * f2 * (a[0] * qa.t[0] + a[1] * qa.t[1] + a[2] * qa.t[2]);
    }

    if (SRC) {
        // dJ/dm_B
        const T v = E0 * f0 + f1 * (E1R + trE2) + f2 * RE2R + f3 * e3.q3 + 3.0 * f2 * e3.Rt;
        out.mB += -G * v + k6 * iA * s4a;
        if (multiB) {
            // dJ/dM2_B = -G [E0 D2 / 2 + (E1 . D3) / 2]
            const T c2 = -0.5 * G * (E0 * f2 + f3 * E1R);
            const T c1 = -0.5 * G * (E0 * f1 + f2 * E1R);
            const T c3 = -0.5 * G * f2;
            out.M2B[0] += c2 * m.xx + c1 + c3 * (2.0 * E1[0] * x);
            out.M2B[1] += c2 * m.xy + c3 * (E1[0] * y + E1[1] * x);
            out.M2B[2] += c2 * m.xz + c3 * (E1[0] * z + E1[2] * x);
            out.M2B[3] += c2 * m.yy + c1 + c3 * (2.0 * E1[1] * y);
            out.M2B[4] += c2 * m.yz + c3 * (E1[1] * z + E1[2] * y);
            out.M2B[5] += c2 * m.zz + c1 + c3 * (2.0 * E1[2] * z);
            // dJ/dM3_B = (G/6) E0 D3 - (G/6) a . D4
            add_rank3(out.M3B, m, a, k6 * (E0 * f3 - f4 * aR), -k6 * f3, k6 * (E0 * f2 - f3 * aR),
                      -k6 * f2);
        }
    }
    if (TGT && useA) {
        // the ratio term -(m_B / m_A) M3_A: dJ/dm_A here; dJ/dM3_A =
        // (G/6) / m_A a . sum_B m_B D4(R_B) from the partners' quartic sum,
        // contracted once per target (reverse_target_finish)
        const T s4 = mB * f4;
        const T txx = s4 * m.xx, txy = s4 * m.xy, txz = s4 * m.xz, tyy = s4 * m.yy, tyz = s4 * m.yz,
                tzz = s4 * m.zz;
        out.A4[0] += txx * m.xx;
        out.A4[1] += txx * m.xy;
        out.A4[2] += txx * m.xz;
        out.A4[3] += txx * m.yy;
        out.A4[4] += txx * m.yz;
        out.A4[5] += txx * m.zz;
        out.A4[6] += txy * m.yy;
        out.A4[7] += txy * m.yz;
        out.A4[8] += txy * m.zz;
        out.A4[9] += txz * m.zz;
        out.A4[10] += tyy * m.yy;
        out.A4[11] += tyy * m.yz;
        out.A4[12] += tyy * m.zz;
        out.A4[13] += tyz * m.zz;
        out.A4[14] += tzz * m.zz;
        out.mA += -k6 * s4a * mB * iA * iA;
    }
    S4Parts<T> m3;  // the partner's octupole parts (interior partners)
    if (want_R) {
        // mB E0 D0 + mB E1.D1 + mB E2:D2 + mB E3:D3
        const T cR = mB * (E0 * f1 + f2 * (E1R + trE2) + f3 * RE2R + f4 * e3.q3 + 3.0 * f3 * e3.Rt);
        T g[3];
#pragma unroll
        for (int p = 0; p < 3; p++)
            g[p] = cR * R[p] + mB * (f1 * E1[p] + 2.0 * f2 * E2R[p] + 3.0 * f3 * e3.q2[p] + 3.0 * f2 * e3.t[p]);
        if (multiB) {
            // E0 M2:D2 / 2 - E0 M3:D3 / 6 + E1 . (D3 : M2) / 2
            T MR[3], ME1[3];
            sym2_vec(M2B, R, MR);
            sym2_vec(M2B, E1, ME1);
            const T xMx = MR[0] * x + MR[1] * y + MR[2] * z;
            const T trM = M2B[0] + M2B[3] + M2B[5];
            const T E1MR = E1[0] * MR[0] + E1[1] * MR[1] + E1[2] * MR[2];
            s4_parts(M3B, m, m3);
            const T cr = 0.5 * E0 * (f3 * xMx + f2 * trM) - (1.0 / 6.0) * E0 * f4 * m3.q3 -
                              0.5 * E0 * f3 * m3.Rt + 0.5 * f4 * E1R * xMx + 0.5 * f3 * (2.0 * E1MR + E1R * trM);
            const T cmr = E0 * f2 + f3 * E1R;
            const T cq2 = -0.5 * E0 * f3, ct = -0.5 * E0 * f2;
            const T ce1 = 0.5 * (f3 * xMx + f2 * trM);
#pragma unroll
            for (int p = 0; p < 3; p++)
                g[p] += cr * R[p] + cmr * MR[p] + cq2 * m3.q2[p] + ct * m3.t[p] + ce1 * E1[p] + f2 * ME1[p];
        }
#pragma unroll
        for (int p = 0; p < 3; p++) gR[p] += -sR * G * g[p];
        if (am && (multiB || useA)) {
            // a . (D4 : Q), Q = M3_B - ratio M3_A
            T Q[10];
#pragma unroll
            for (int n = 0; n < 10; n++) Q[n] = (multiB ? M3B[n] : 0.0) - (useA ? ratio * M3A[n] : 0.0);
            // the parts of Q are linear in Q: from the octupoles' own parts
            S4Parts<T> q;
            const T rq = useA ? ratio : T(0.0);
#pragma unroll
            for (int p = 0; p < 3; p++) {
                q.q2[p] = (multiB ? m3.q2[p] : T(0.0)) - (useA ? rq * qa.q2[p] : T(0.0));
                q.t[p] = (multiB ? m3.t[p] : T(0.0)) - (useA ? rq * qa.t[p] : T(0.0));
            }
            q.q3 = (multiB ? m3.q3 : T(0.0)) - (useA ? rq * qa.q3 : T(0.0));
            q.Rt = (multiB ? m3.Rt : T(0.0)) - (useA ? rq * qa.Rt : T(0.0));
            T u[3];  // u_p = Q_pik a_i R_k
            sym3_contract(Q, a[0] * x, a[1] * y, a[2] * z, a[0] * y + a[1] * x, a[0] * z + a[2] * x,
                          a[1] * z + a[2] * y, u);
            const T aq2 = a[0] * q.q2[0] + a[1] * q.q2[1] + a[2] * q.q2[2];
            const T at = a[0] * q.t[0] + a[1] * q.t[1] + a[2] * q.t[2];
            const T cv = f5 * aR * q.q3 + 3.0 * f4 * aq2 + 3.0 * f4 * aR * q.Rt + 3.0 * f3 * at;
            const T ca = f4 * q.q3 + 3.0 * f3 * q.Rt;
#pragma unroll
            for (int p = 0; p < 3; p++)
                gR[p] += -sR * k6 * (cv * R[p] + ca * a[p] + 3.0 * f4 * aR * q.q2[p] + 6.0 * f3 * u[p] +
                                        3.0 * f3 * aR * q.t[p]);
        }
    }
}


// dJ/dM3_A of a target from the quartic sum A4 = sum_B m_B f4 R^4 that the
// target's pairs accumulated: dJ/dM3_A = (G/6) / m_A a . sum_B m_B D4(R_B),
// where sum m D4 = A4 + sym(delta Q) + c0 sym(delta delta) with Q = sum m f3
// R R = -tr(A4) / 7 and c0 = sum m f2 = -tr(Q) / 5 (D4 is traceless); so per
// packed jkl: (a.A4)_jkl + a_j Q_kl + a_k Q_jl + a_l Q_jk + delta_jk (Q a)_l
// + delta_jl (Q a)_k + delta_kl (Q a)_j + c0 (a_j delta_kl + a_k delta_jl
// + a_l delta_jk).  kr = (G/6) / m_A.
template <class T>
__host__ __device__ __forceinline__ void reverse_target_finish(PairAdjOutT<T>& o, const T* a, T kr) {
    const T* q = o.A4;  // xxxx xxxy xxxz xxyy xxyz xxzz xyyy xyyz xyzz xzzz yyyy yyyz yyzz yzzz zzzz
    const T s7 = T(-1.0 / 7.0);
    const T Qxx = s7 * (q[0] + q[3] + q[5]), Qxy = s7 * (q[1] + q[6] + q[8]);
    const T Qxz = s7 * (q[2] + q[7] + q[9]), Qyy = s7 * (q[3] + q[10] + q[12]);
    const T Qyz = s7 * (q[4] + q[11] + q[13]), Qzz = s7 * (q[5] + q[12] + q[14]);
    const T c0 = T(-0.2) * (Qxx + Qyy + Qzz);
    const T Qa[3] = {Qxx * a[0] + Qxy * a[1] + Qxz * a[2], Qxy * a[0] + Qyy * a[1] + Qyz * a[2],
                     Qxz * a[0] + Qyz * a[1] + Qzz * a[2]};
    // (a . A4)_jkl for the packed rank-3 jkl: sum_i a_i A4_ijkl
    const T aA[10] = {
        a[0] * q[0] + a[1] * q[1] + a[2] * q[2],     // xxx
        a[0] * q[1] + a[1] * q[3] + a[2] * q[4],     // xxy
        a[0] * q[2] + a[1] * q[4] + a[2] * q[5],     // xxz
        a[0] * q[3] + a[1] * q[6] + a[2] * q[7],     // xyy
        a[0] * q[4] + a[1] * q[7] + a[2] * q[8],     // xyz
        a[0] * q[5] + a[1] * q[8] + a[2] * q[9],     // xzz
        a[0] * q[6] + a[1] * q[10] + a[2] * q[11],   // yyy
        a[0] * q[7] + a[1] * q[11] + a[2] * q[12],   // yyz
        a[0] * q[8] + a[1] * q[12] + a[2] * q[13],   // yzz
        a[0] * q[9] + a[1] * q[13] + a[2] * q[14]};  // zzz
    const T Q2[3][3] = {{Qxx, Qxy, Qxz}, {Qxy, Qyy, Qyz}, {Qxz, Qyz, Qzz}};
    const int P3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                           {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
#pragma unroll
    for (int n = 0; n < 10; n++) {
        const int j = P3[n][0], k = P3[n][1], l = P3[n][2];
        T v = aA[n] + a[j] * Q2[k][l] + a[k] * Q2[j][l] + a[l] * Q2[j][k];
        if (j == k) v += Qa[l] + c0 * a[l];
        if (j == l) v += Qa[k] + c0 * a[k];
        if (k == l) v += Qa[j] + c0 * a[j];
        o.M3A[n] += kr * v;
    }
}

}  // namespace otfmm
