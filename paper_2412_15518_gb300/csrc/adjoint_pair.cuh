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

#include "pair_formula.cuh"

namespace otfmm {

template <class T> struct PairAdjOutT {
    T mB, M2B[6], M3B[10];
    T mA, M3A[10];
    T R[3];
    T A4[15];  // target side: sum over partners of m_B f4 R^4 (reverse_target_quartic;
               // reverse_target_finish)
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

// What the reverse pair needs of its target that does not depend on the
// partner, formed once per target (reverse_target_prep) instead of per pair:
// e0 / 2 and -e0 / 6; for an interior target (EFULL) the trace of E2 and
// three times the trace vector of E3 (E3_ijj); for the correction's mass
// ratio (useA) the trace vector of M3A, a . that vector and 1 / m_A^2.
template <class T> struct RevTarget {
    T he0, e6;
    T trE2, te3[3];
    T ta[3], ata, iA2;
};

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

template <bool EFULL, class T>
__host__ __device__ __forceinline__ void reverse_target_prep(T e0, const T* e2, const T* e3, bool useA,
                                                             T iA, const T* M3A, const T* a,
                                                             RevTarget<T>& tg) {
    tg.he0 = T(0.5) * e0;
    tg.e6 = T(-1.0 / 6.0) * e0;
    tg.trE2 = T(0.0);
    tg.ata = T(0.0);
    tg.iA2 = T(0.0);
#pragma unroll
    for (int p = 0; p < 3; p++) {
        tg.te3[p] = T(0.0);
        tg.ta[p] = T(0.0);
    }
    if (EFULL) {
        tg.trE2 = e2[0] + e2[3] + e2[5];
        T te[3];
        sym3_trace(e3, te);
#pragma unroll
        for (int p = 0; p < 3; p++) tg.te3[p] = T(3.0) * te[p];
    }
    if (useA) {
        sym3_trace(M3A, tg.ta);
        tg.ata = fma_(a[0], tg.ta[0], fma_(a[1], tg.ta[1], a[2] * tg.ta[2]));
        tg.iA2 = iA * iA;
    }
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

// Reverse of one pair, added into out, without the -G factors and in the
// caller's units.  By homogeneity the pair's physical expansion is
// -G h^-(n+1) times its value from R' = R / h, M2' = M2 / h^2, M3' = M3 / h^3
// (and the correction -(G/6) h^-2 times D4(R') : Q'), so the caller passes R
// and the moments in cell units and the adjoints pre-scaled,
//   e0 = -G h^-1 E0, e1 = -G h^-2 E1, e2 = -G h^-3 E2, e3 = -G h^-4 E3,
//   al = -(G/6) h^-2 a,
// and receives dJ/dm_B and dJ/dm_A in physical units, dJ/dM2_B, dJ/dM3_B and
// dJ/dR times oM2, oM3 and oR (h^-2, h^-3 and +-h^-1 give physical adjoints,
// the sign that of the centre of mass that R moves).  With h = 1 and G
// folded into the adjoints this is the physical pair.
//   SRC: the source's adjoints (m_B; M2_B, M3_B for an interior source,
//        multiB, whose trace vector M3_B,ijj and trace of M2_B come in btB),
//        added to out.mB, out.M2B, out.M3B;
//   TGT: the target side of the correction's mass ratio (useA: an interior
//        target of mass m_A = 1 / iA != 0, octupole M3A): out.mA; the
//        quartic sum out.A4 = sum_B m_B f4 R^4 that reverse_target_finish
//        needs is the forward pair's own (reverse_target_quartic);
//   EFULL: the target has E2 and E3 adjoints (an interior target; a leaf
//        target's are zero and skipped);
//   want_R: dJ/dR into gR.
// tg holds the target's partner-independent parts (reverse_target_prep with
// the same e0, e2, e3, useA, iA, M3A and al).
template <bool SRC, bool TGT, bool EFULL, class T>
__host__ __device__ __forceinline__ void m2l_pair_reverse(
    const T* Rv, T mB, const T* M2B, const T* M3B, const T* btB, bool multiB, bool useA, T iA,
    const T* M3A, T e0, const T* e1, const T* e2, const T* e3, const RevTarget<T>& tg, bool am,
    const T* al, bool want_R, T oM2, T oM3, T oR, T* gR, PairAdjOutT<T>& out) {
    const T x = Rv[0], y = Rv[1], z = Rv[2];
    const T R[3] = {x, y, z};
    const T xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    const T xy2 = xy + xy, xz2 = xz + xz, yz2 = yz + yz;
    const T f0 = rsqrt_adj(xx + yy + zz);
    const T ri2 = f0 * f0;
    const T f1 = -(f0 * ri2);
    const T f2 = f1 * (T(-3.0) * ri2);
    const T f3 = f2 * (T(-5.0) * ri2);
    const T f4 = f3 * (T(-7.0) * ri2);
    const T zero3[3] = {T(0.0), T(0.0), T(0.0)};
    const T* a = am ? al : zero3;
    const T aR = fma_(a[0], x, fma_(a[1], y, a[2] * z));
    const T e1R = fma_(e1[0], x, fma_(e1[1], y, e1[2] * z));

    // the interior target's E2 and E3 with R: e2R = E2 R, Re2R = R.E2.R,
    // q2e = E3 : R R, q3e = R.q2e, te = the trace vector of E3 (3 te in
    // tg.te3), Rte = R.te; sum1 = e1R + tr E2 and sum2 = Re2R + 3 Rte recur
    // below
    T e2R[3] = {T(0.0), T(0.0), T(0.0)}, q2e[3] = {T(0.0), T(0.0), T(0.0)};
    T q3e = T(0.0), sum1 = e1R, sum2 = T(0.0);
    if (EFULL) {
        e2R[0] = fma_(e2[0], x, fma_(e2[1], y, e2[2] * z));
        e2R[1] = fma_(e2[1], x, fma_(e2[3], y, e2[4] * z));
        e2R[2] = fma_(e2[2], x, fma_(e2[4], y, e2[5] * z));
        const T Re2R = fma_(x, e2R[0], fma_(y, e2R[1], z * e2R[2]));
        sum1 = e1R + tg.trE2;
        contract_rr(e3, xx, yy, zz, xy2, xz2, yz2, q2e[0], q2e[1], q2e[2]);
        q3e = fma_(x, q2e[0], fma_(y, q2e[1], z * q2e[2]));
        sum2 = fma_(x, tg.te3[0], fma_(y, tg.te3[1], fma_(z, tg.te3[2], Re2R)));
    }
    // the target octupole's parts (the correction's ratio term) and
    // s4a = a . (D4 : M3A)
    T q2a[3] = {T(0.0), T(0.0), T(0.0)};
    T q3a = T(0.0), Rta = T(0.0), s4a = T(0.0);
    const T f4aR = f4 * aR;
    if (useA) {
        contract_rr(M3A, xx, yy, zz, xy2, xz2, yz2, q2a[0], q2a[1], q2a[2]);
        q3a = fma_(x, q2a[0], fma_(y, q2a[1], z * q2a[2]));
        Rta = fma_(x, tg.ta[0], fma_(y, tg.ta[1], z * tg.ta[2]));
        const T aq2a = fma_(a[0], q2a[0], fma_(a[1], q2a[1], a[2] * q2a[2]));
        s4a = fma_(f4aR, q3a, T(3.0) * fma_(f3, fma_(aR, Rta, aq2a), f2 * tg.ata));
    }

    if (SRC) {
        // dJ/dm_B = e0 D0 + e1.D1 + e2:D2 + e3:D3 - a.(D4:M3A) / m_A
        T v = fma_(f1, sum1, e0 * f0);
        if (EFULL) v = fma_(f2, sum2, fma_(f3, q3e, v));
        if (useA) v = fma_(-iA, s4a, v);
        out.mB += v;
        if (multiB) {
            // dJ/dM2_B = [e0 D2 + e1 . D3] / 2
            //   = [(e0 f2 + f3 e1R) R R + (e0 f1 + f2 e1R) I + f2 (e1 R + R e1)] / 2
            const T h = T(0.5) * oM2;
            const T c2 = h * fma_(e0, f2, f3 * e1R);
            const T c1 = h * fma_(e0, f1, f2 * e1R);
            const T c3 = h * f2;
            const T ex = c3 * e1[0], ey = c3 * e1[1], ez = c3 * e1[2];
            out.M2B[0] = fma_(c2, xx, fma_(ex + ex, x, out.M2B[0] + c1));
            out.M2B[1] = fma_(c2, xy, fma_(ex, y, fma_(ey, x, out.M2B[1])));
            out.M2B[2] = fma_(c2, xz, fma_(ex, z, fma_(ez, x, out.M2B[2])));
            out.M2B[3] = fma_(c2, yy, fma_(ey + ey, y, out.M2B[3] + c1));
            out.M2B[4] = fma_(c2, yz, fma_(ey, z, fma_(ez, y, out.M2B[4])));
            out.M2B[5] = fma_(c2, zz, fma_(ez + ez, z, out.M2B[5] + c1));
            // dJ/dM3_B = -e0 D3 / 6 + a . D4
            //   = k4 RRR + k3 (aRR) + k3r (IR) + k2 (Ia), with
            // (aRR)_jkl = a_j R_k R_l + a_k R_j R_l + a_l R_j R_k, (IR)_jkl =
            // d_jk R_l + d_jl R_k + d_kl R_j and (Ia) likewise with a
            const T k4 = oM3 * fma_(tg.e6, f3, f4aR);
            const T k3r = oM3 * fma_(f3, aR, tg.e6 * f2);
            const T k3 = oM3 * f3, k2 = oM3 * f2;
            const T ax = k3 * a[0], ay = k3 * a[1], az = k3 * a[2];
            const T bx = k2 * a[0], by = k2 * a[1], bz = k2 * a[2];
            const T kx = k4 * x, ky = k4 * y, kz = k4 * z;
            T* o = out.M3B;
            o[0] = fma_(kx, xx, fma_(T(3.0), fma_(ax, xx, fma_(k3r, x, bx)), o[0]));   // xxx
            o[1] = fma_(kx, xy, fma_(ax, xy2, fma_(ay, xx, fma_(k3r, y, by + o[1])))); // xxy
            o[2] = fma_(kx, xz, fma_(ax, xz2, fma_(az, xx, fma_(k3r, z, bz + o[2])))); // xxz
            o[3] = fma_(kx, yy, fma_(ax, yy, fma_(ay, xy2, fma_(k3r, x, bx + o[3])))); // xyy
            o[4] = fma_(kx, yz, fma_(ax, yz, fma_(ay, xz, fma_(az, xy, o[4]))));       // xyz
            o[5] = fma_(kx, zz, fma_(ax, zz, fma_(az, xz2, fma_(k3r, x, bx + o[5])))); // xzz
            o[6] = fma_(ky, yy, fma_(T(3.0), fma_(ay, yy, fma_(k3r, y, by)), o[6]));   // yyy
            o[7] = fma_(ky, yz, fma_(ay, yz2, fma_(az, yy, fma_(k3r, z, bz + o[7])))); // yyz
            o[8] = fma_(ky, zz, fma_(ay, zz, fma_(az, yz2, fma_(k3r, y, by + o[8])))); // yzz
            o[9] = fma_(kz, zz, fma_(T(3.0), fma_(az, zz, fma_(k3r, z, bz)), o[9]));   // zzz
        }
    }
    if (TGT && useA) {
        // the ratio term -(m_B / m_A) M3A: dJ/dm_A = m_B / m_A^2 a.(D4:M3A)
        // here; dJ/dM3_A = -(1 / m_A) a . sum_B m_B D4(R_B) once per target
        // (reverse_target_finish)
        out.mA = fma_(mB * tg.iA2, s4a, out.mA);
    }
    if (!want_R) return;
    // dJ/dR: the monopole part mB (e0 D1 + e1.D2 + e2:D3 + e3:D4)
    T g[3];
    {
        const T a1 = mB * f1;
        if (EFULL) {
            const T cR = mB * fma_(e0, f1, fma_(f2, sum1, fma_(f3, sum2, f4 * q3e)));
            const T a2 = mB * f2, a3 = T(3.0) * (mB * f3);
#pragma unroll
            for (int p = 0; p < 3; p++)
                g[p] = fma_(cR, R[p], fma_(a1, e1[p], fma_(a2, fma_(T(2.0), e2R[p], tg.te3[p]),
                                                            a3 * q2e[p])));
        } else {
            const T cR = mB * fma_(e0, f1, f2 * e1R);
#pragma unroll
            for (int p = 0; p < 3; p++) g[p] = fma_(cR, R[p], a1 * e1[p]);
        }
    }
    // the source octupole's parts (interior sources; its trace vector tb
    // comes in btB)
    T q2b[3] = {T(0.0), T(0.0), T(0.0)}, q3b = T(0.0), Rtb = T(0.0);
    const T* tb = btB;
    if (multiB) {
        // e0 (M2:D2 / 2 - M3:D3 / 6) + e1 . (D3 : M2) / 2
        T MR[3], ME1[3];
        MR[0] = fma_(M2B[0], x, fma_(M2B[1], y, M2B[2] * z));
        MR[1] = fma_(M2B[1], x, fma_(M2B[3], y, M2B[4] * z));
        MR[2] = fma_(M2B[2], x, fma_(M2B[4], y, M2B[5] * z));
        ME1[0] = fma_(M2B[0], e1[0], fma_(M2B[1], e1[1], M2B[2] * e1[2]));
        ME1[1] = fma_(M2B[1], e1[0], fma_(M2B[3], e1[1], M2B[4] * e1[2]));
        ME1[2] = fma_(M2B[2], e1[0], fma_(M2B[4], e1[1], M2B[5] * e1[2]));
        const T xMx = fma_(x, MR[0], fma_(y, MR[1], z * MR[2]));
        const T trM = btB[3];
        const T E1MR = fma_(e1[0], MR[0], fma_(e1[1], MR[1], e1[2] * MR[2]));
        contract_rr(M3B, xx, yy, zz, xy2, xz2, yz2, q2b[0], q2b[1], q2b[2]);
        q3b = fma_(x, q2b[0], fma_(y, q2b[1], z * q2b[2]));
        Rtb = fma_(x, tb[0], fma_(y, tb[1], z * tb[2]));
        const T he0 = tg.he0;
        const T A2 = fma_(f3, xMx, f2 * trM);  // f3 xMx + f2 trM
        const T B2 = fma_(f4, xMx, f3 * trM);  // f4 xMx + f3 trM
        // R_p: e0 [(f3 xMx + f2 trM) / 2 - f4 q3 / 6 - f3 Rt / 2]
        //      + e1R (f4 xMx + f3 trM) / 2 + f3 e1.M2 R
        const T cr = fma_(he0, fma_(-f3, Rtb, fma_(T(-1.0 / 3.0) * f4, q3b, A2)),
                          fma_(T(0.5) * e1R, B2, f3 * E1MR));
        const T cmr = fma_(e0, f2, f3 * e1R);
        const T cq2 = -(he0 * f3), ct = -(he0 * f2), ce1 = T(0.5) * A2;
#pragma unroll
        for (int p = 0; p < 3; p++)
            g[p] = fma_(cr, R[p], fma_(cmr, MR[p], fma_(cq2, q2b[p], fma_(ct, tb[p], fma_(ce1, e1[p],
                                                                                     fma_(f2, ME1[p], g[p]))))));
    }
    if (am && (multiB || useA)) {
        // a . grad_R (D4 : Q), Q = M3_B - (m_B / m_A) M3A: the parts of Q are
        // those of the two octupoles combined
        T q2[3], tq[3], Q[10], q3 = q3b, Rt = Rtb;
#pragma unroll
        for (int p = 0; p < 3; p++) {
            q2[p] = q2b[p];
            tq[p] = multiB ? tb[p] : T(0.0);
        }
#pragma unroll
        for (int n = 0; n < 10; n++) Q[n] = M3B[n];
        if (useA) {
            const T rq = mB * iA;
#pragma unroll
            for (int p = 0; p < 3; p++) {
                q2[p] = fma_(-rq, q2a[p], q2[p]);
                tq[p] = fma_(-rq, tg.ta[p], tq[p]);
            }
            q3 = fma_(-rq, q3a, q3);
            Rt = fma_(-rq, Rta, Rt);
#pragma unroll
            for (int n = 0; n < 10; n++) Q[n] = fma_(-rq, M3A[n], Q[n]);
        }
        T u[3];  // u_p = Q_pik a_i R_k
        sym3_contract(Q, a[0] * x, a[1] * y, a[2] * z, fma_(a[0], y, a[1] * x), fma_(a[0], z, a[2] * x),
                      fma_(a[1], z, a[2] * y), u);
        const T aq2 = fma_(a[0], q2[0], fma_(a[1], q2[1], a[2] * q2[2]));
        const T at = fma_(a[0], tq[0], fma_(a[1], tq[1], a[2] * tq[2]));
        const T f5 = f4 * (T(-9.0) * ri2);
        const T F3 = T(3.0) * f3;
        // R_p: f5 aR q3 + 3 f4 (a.q2 + aR Rt) + 3 f3 a.t; a_p: f4 q3 + 3 f3 Rt
        const T cv = fma_(f5 * aR, q3, fma_(T(3.0) * f4, fma_(aR, Rt, aq2), F3 * at));
        const T ca = fma_(f4, q3, F3 * Rt);
        const T cq = T(3.0) * f4aR, cu = F3 + F3, ctq = F3 * aR;
#pragma unroll
        for (int p = 0; p < 3; p++)
            g[p] = fma_(cv, R[p], fma_(ca, a[p], fma_(cq, q2[p], fma_(cu, u[p], fma_(ctq, tq[p], g[p])))));
    }
#pragma unroll
    for (int p = 0; p < 3; p++) gR[p] = fma_(oR, g[p], gR[p]);
}


// The target's quartic sum A4 += m_B f4 R^4 of one pair (R from the target):
// the forward pair's own sum (pair_formula.cuh, Acc::A4 times kAccCor), which
// the adjoint's forward pass keeps per interior target; every quartic
// monomial is a square's multiple times a quadratic one.
template <class T>
__host__ __device__ __forceinline__ void reverse_target_quartic(const T* Rv, T mB, PairAdjOutT<T>& out) {
    const T x = Rv[0], y = Rv[1], z = Rv[2];
    const T xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    const T f0 = rsqrt_adj(xx + yy + zz);
    const T ri2 = f0 * f0;
    const T f4 = T(105.0) * (f0 * ri2 * ri2 * ri2 * ri2);
    const T s4 = mB * f4;
    const T txx = s4 * xx, tyy = s4 * yy, tzz = s4 * zz;
    out.A4[0] = fma_(txx, xx, out.A4[0]);
    out.A4[1] = fma_(txx, xy, out.A4[1]);
    out.A4[2] = fma_(txx, xz, out.A4[2]);
    out.A4[3] = fma_(txx, yy, out.A4[3]);
    out.A4[4] = fma_(txx, yz, out.A4[4]);
    out.A4[5] = fma_(txx, zz, out.A4[5]);
    out.A4[6] = fma_(tyy, xy, out.A4[6]);
    out.A4[7] = fma_(tyy, xz, out.A4[7]);
    out.A4[8] = fma_(tzz, xy, out.A4[8]);
    out.A4[9] = fma_(tzz, xz, out.A4[9]);
    out.A4[10] = fma_(tyy, yy, out.A4[10]);
    out.A4[11] = fma_(tyy, yz, out.A4[11]);
    out.A4[12] = fma_(tyy, zz, out.A4[12]);
    out.A4[13] = fma_(tzz, yz, out.A4[13]);
    out.A4[14] = fma_(tzz, zz, out.A4[14]);
}

// dJ/dM3_A of a target from the quartic sum A4 = sum_B m_B f4 R^4 over the
// target's pairs: dJ/dM3_A = (G/6) / m_A a . sum_B m_B D4(R_B),
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
