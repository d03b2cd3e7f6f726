// One cell-to-cell multipole interaction (M2L of total order 3 plus the
// angular-momentum correction), written once as a template over the scalar
// type: double for the FP64 form, float for the FP32-bulk form, and a
// counting type on the host for the flop accounting of the roofline.
//
// Reading of the paper (Sec. 4.3.1: the FMM conserves linear momentum and,
// through a special technique, angular momentum):
//   R = X_A - X_B, D^(n) = grad^n (1/|R|);
//   L^(n)_A += -G sum_{m <= 3-n} (-1)^m / m!  M^(m)_B ._m D^(n+m)(R)
//   a_c,A   += -(G/6) D^(4)(R) ._3 [M3_B - (m_B / m_A) M3_A]
//            = -(G/6) [S - P],  S = sum_B D4 ._3 M3_B,
//                               P = (sum_B m_B D4) ._3 (M3_A / m_A)
// The target octupole per unit mass is fixed for a target, so P is formed
// once per target (correction_target) from the sum A4 = sum_B m_B f4 R^4 of
// the pairs' pure quartic parts: D4 is traceless, so its lower parts follow
// from A4's traces (sum m f3 R R = -tr A4 / 7, sum m f2 = tr tr A4 / 35).
// With f_k = (-1)^k (2k-1)!! / r^(2k+1), every contraction of a symmetric
// tensor with D^(n) reduces to a few scalars: for S = M2 (Mx = M2 R,
// xMx = R.M2.R, tr = trace) and T = M3 (q2 = T:RR, q3 = R.q2, t_i = T_ijj,
// Rt = R.t):
//   M2 : D2        = f2 xMx + f1 tr
//   (D3 . M2)_i    = f3 R_i xMx + f2 (2 Mx_i + R_i tr)
//   M3 : D3        = f3 q3 + 3 f2 Rt
//   (D4 : M3)_i    = f4 R_i q3 + 3 f3 (q2_i + R_i Rt) + 3 f2 t_i
// so no D tensor is ever formed.  Everything here is in units of the cell
// side h (R' = R / h, M2' = M2 / h^2, M3' = M3 / h^3) and without the -G
// factor; the caller scales L^(n) by -G h^-(n+1) and the correction sums S
// and P by -(G/6) h^-2 once per target.
//
// The radial factors are formed as the plain chain g_k = 1/r^(2k+1)
// (f_k = (-1)^k (2k-1)!! g_k): the constants of the monopole sums L2, L3 and
// A4 and of the correction sum S are left out of the per-pair work and
// applied once per target with the level's scale factors (kAccL2, kAccL3,
// kAccCor below).
#pragma once

#include "common.cuh"

namespace otfmm {

template <class T> struct Acc {
    T L0, L1[3];
    T L2[6];  // sum m g2 R R = L2 / kAccL2 (before finish_acc)
    T L3[10]; // sum m g3 R R R = L3 / kAccL3 (before finish_acc)
    T S[3];   // correction sum of the source octupoles / kAccCor
    T A4[15]; // sum m_B g4 R^4 = sum m_B f4 R^4 / kAccCor of interior targets (xxxx
              // xxxy xxxz xxyy xxyz xxzz xyyy xyyz xyzz xzzz yyyy yyyz yyzz yzzz zzzz)
};
// The constants left out of the sums: f2 = 3 g2, f3 = -15 g3, f4 = 105 g4.
// finish_acc and correction_target are linear, so they act on the sums as
// held; the flush multiplies the level's scale of L2 by kAccL2, of L3 by
// kAccL3 and of the correction (S - P) by kAccCor.
constexpr double kAccL2 = 3.0, kAccL3 = -15.0, kAccCor = 105.0;
// The Kronecker parts of L2 and L3 are not accumulated: D2 and D3 are
// traceless, so per pair sum m f1 = -trace(m f2 R R) / 3 and
// sum m f2 R = -trace(m f3 R R R) / 5; finish_acc restores them from the
// accumulated R R and R R R parts once per target.

template <class T> __host__ __device__ __forceinline__ void acc_zero(Acc<T>& A) {
    A.L0 = T(0.0);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        A.L1[i] = T(0.0);
        A.S[i] = T(0.0);
    }
#pragma unroll
    for (int i = 0; i < 15; i++) A.A4[i] = T(0.0);
#pragma unroll
    for (int i = 0; i < 6; i++) A.L2[i] = T(0.0);
#pragma unroll
    for (int i = 0; i < 10; i++) A.L3[i] = T(0.0);
}

// Adds the Kronecker parts to L2 (d1 on the diagonal) and L3 (delta_ij V_k
// + delta_ik V_j + delta_jk V_i), d1 and V taken from the traces.
template <class T> __host__ __device__ __forceinline__ void finish_acc(Acc<T>& A) {
    const T d1 = T(-1.0 / 3.0) * (A.L2[0] + A.L2[3] + A.L2[5]);
    const T Vx = T(-0.2) * (A.L3[0] + A.L3[3] + A.L3[5]);
    const T Vy = T(-0.2) * (A.L3[1] + A.L3[6] + A.L3[8]);
    const T Vz = T(-0.2) * (A.L3[2] + A.L3[7] + A.L3[9]);
    A.L2[0] += d1;
    A.L2[3] += d1;
    A.L2[5] += d1;
    A.L3[0] += T(3.0) * Vx;
    A.L3[1] += Vy;
    A.L3[2] += Vz;
    A.L3[3] += Vx;
    A.L3[5] += Vx;
    A.L3[6] += T(3.0) * Vy;
    A.L3[7] += Vz;
    A.L3[8] += Vy;
    A.L3[9] += T(3.0) * Vz;
}

__host__ __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
#ifdef __CUDA_ARCH__
__device__ __forceinline__ double rsqrt_(double a) { return rsqrt(a); }
// FP32: the hardware reciprocal square root is an approximation whose error
// is a smooth function of R, so it does not average out over pairs and the
// D-tensor factors f_k ~ f0^(2k+1) amplify it.  One Newton-Raphson step,
// y <- y + y (1 - a y^2) / 2 with the residual formed by an FMA, brings the
// seed to about an ulp.
__device__ __forceinline__ float rsqrt_(float a) {
    const float y = rsqrtf(a);
    return fmaf(0.5f * y, fmaf(-a * y, y, 1.0f), y);
}
#else
inline double rsqrt_(double a) { return 1.0 / sqrt(a); }
inline float rsqrt_(float a) { return 1.0f / sqrtf(a); }
#endif

// q2 = T : R R for a packed symmetric rank-3 tensor (xxx xxy xxz xyy xyz xzz
// yyy yyz yzz zzz), given the six products with the off-diagonal ones doubled.
template <class T>
__host__ __device__ __forceinline__ void contract_rr(const T* c, T xx, T yy, T zz, T xy2, T xz2,
                                                     T yz2, T& qx, T& qy, T& qz) {
    qx = fma_(c[0], xx, fma_(c[3], yy, fma_(c[5], zz, fma_(c[1], xy2, fma_(c[2], xz2, c[4] * yz2)))));
    qy = fma_(c[1], xx, fma_(c[6], yy, fma_(c[8], zz, fma_(c[3], xy2, fma_(c[4], xz2, c[7] * yz2)))));
    qz = fma_(c[2], xx, fma_(c[7], yy, fma_(c[9], zz, fma_(c[4], xy2, fma_(c[5], xz2, c[8] * yz2)))));
}

// The target part of the correction, P_i = sum_jkl (sum m D4)_ijkl a_jkl,
// from A4 with a = M3' / m_A (packed) and t its trace vector:
//   P = A4 : a + 3 Q : a + 3 Q t + 3 c0 t,  Q = -tr A4 / 7,  c0 = tr tr A4 / 35.
template <class T>
__host__ __device__ __forceinline__ void correction_target(const Acc<T>& A, const T* a, const T* t,
                                                           T* P) {
    const T* q = A.A4;
    const T s7 = T(-1.0 / 7.0);
    const T Qxx = s7 * (q[0] + q[3] + q[5]), Qxy = s7 * (q[1] + q[6] + q[8]);
    const T Qxz = s7 * (q[2] + q[7] + q[9]), Qyy = s7 * (q[3] + q[10] + q[12]);
    const T Qyz = s7 * (q[4] + q[11] + q[13]), Qzz = s7 * (q[5] + q[12] + q[14]);
    const T c0 = T(1.0 / 35.0) * (q[0] + q[10] + q[14] + T(2.0) * (q[3] + q[5] + q[12]));
    // a weighted by the multiplicity of its packed index in a full contraction
    const T w[10] = {a[0], T(3.0) * a[1], T(3.0) * a[2], T(3.0) * a[3], T(6.0) * a[4],
                     T(3.0) * a[5], a[6], T(3.0) * a[7], T(3.0) * a[8], a[9]};
    const T Ax = q[0] * w[0] + q[1] * w[1] + q[2] * w[2] + q[3] * w[3] + q[4] * w[4] + q[5] * w[5] +
                 q[6] * w[6] + q[7] * w[7] + q[8] * w[8] + q[9] * w[9];
    const T Ay = q[1] * w[0] + q[3] * w[1] + q[4] * w[2] + q[6] * w[3] + q[7] * w[4] + q[8] * w[5] +
                 q[10] * w[6] + q[11] * w[7] + q[12] * w[8] + q[13] * w[9];
    const T Az = q[2] * w[0] + q[4] * w[1] + q[5] * w[2] + q[7] * w[3] + q[8] * w[4] + q[9] * w[5] +
                 q[11] * w[6] + q[12] * w[7] + q[13] * w[8] + q[14] * w[9];
    T Qax, Qay, Qaz;
    contract_rr(a, Qxx, Qyy, Qzz, Qxy + Qxy, Qxz + Qxz, Qyz + Qyz, Qax, Qay, Qaz);
    const T Qtx = Qxx * t[0] + Qxy * t[1] + Qxz * t[2];
    const T Qty = Qxy * t[0] + Qyy * t[1] + Qyz * t[2];
    const T Qtz = Qxz * t[0] + Qyz * t[1] + Qzz * t[2];
    P[0] = Ax + T(3.0) * (Qax + Qtx + c0 * t[0]);
    P[1] = Ay + T(3.0) * (Qay + Qty + c0 * t[1]);
    P[2] = Az + T(3.0) * (Qaz + Qtz + c0 * t[2]);
}

// TGT_FULL: the target is an interior cell (needs L2, L3 and the target part
// of the correction).  SRC_MULTI: the source is an interior cell (has M2, M3).
// AM: the correction is on.  (x, y, z) = R', m = source mass, b2/b3 = source
// M2'/M3', bt = the source's M3 trace vector (t_i = M3_ijj) and trace of M2
// (bt[3]).
template <class T, bool TGT_FULL, bool SRC_MULTI, bool AM>
__host__ __device__ __forceinline__ void m2l_pair(T x, T y, T z, T m, const T* b2, const T* b3,
                                                  const T* bt, Acc<T>& A) {
    constexpr bool kHigh = TGT_FULL || SRC_MULTI;  // needs g2 and g3
    const T r2 = fma_(x, x, fma_(y, y, z * z));
    const T g0 = rsqrt_(r2);
    const T ri2 = g0 * g0;
    const T g1 = g0 * ri2;
    T g2 = T(0.0), g3 = T(0.0), g4 = T(0.0);
    if (kHigh) {
        g2 = g1 * ri2;
        g3 = g2 * ri2;
    }
    if (kHigh && AM) g4 = g3 * ri2;
    const T c1 = m * g1;  // -m f1
    T xx = T(0.0), yy = T(0.0), zz = T(0.0), xy = T(0.0), xz = T(0.0), yz = T(0.0);
    if (kHigh) {
        xx = x * x;
        yy = y * y;
        zz = z * z;
        xy = x * y;
        xz = x * z;
        yz = y * z;
    }
    if (SRC_MULTI) {
        const T xy2 = xy + xy, xz2 = xz + xz, yz2 = yz + yz;
        const T Mx = fma_(b2[0], x, fma_(b2[1], y, b2[2] * z));
        const T My = fma_(b2[1], x, fma_(b2[3], y, b2[4] * z));
        const T Mz = fma_(b2[2], x, fma_(b2[4], y, b2[5] * z));
        const T xMx = fma_(x, Mx, fma_(y, My, z * Mz));
        const T tr = bt[3];
        T qx, qy, qz;
        contract_rr(b3, xx, yy, zz, xy2, xz2, yz2, qx, qy, qz);
        const T q3 = fma_(x, qx, fma_(y, qy, z * qz));
        const T Rt = fma_(x, bt[0], fma_(y, bt[1], z * bt[2]));
        const T h2 = T(1.5) * g2;  // f2 / 2
        // L0 += m f0 + (f2 xMx + f1 tr) / 2 - (f3 q3 + 3 f2 Rt) / 6
        //     = m g0 - g1 tr / 2 + (3/2) g2 (xMx - Rt) + (5/2) g3 q3
        A.L0 = fma_(m, g0, fma_(T(-0.5) * g1, tr, fma_(h2, xMx - Rt, fma_(T(2.5) * g3, q3, A.L0))));
        // L1 += R (m f1 + (f3 xMx + f2 tr) / 2) + f2 M2 R
        //     = R (-m g1 - (15/2) g3 xMx + (3/2) g2 tr) + 3 g2 M2 R
        const T e = fma_(T(-7.5) * g3, xMx, fma_(h2, tr, -c1));
        const T d2 = h2 + h2;
        A.L1[0] = fma_(e, x, fma_(d2, Mx, A.L1[0]));
        A.L1[1] = fma_(e, y, fma_(d2, My, A.L1[1]));
        A.L1[2] = fma_(e, z, fma_(d2, Mz, A.L1[2]));
        if (AM) {
            // S += f4 R q3 + 3 f3 (q2 + R Rt) + 3 f2 t, held / 105:
            //    R (g4 q3 - (3/7) g3 Rt) - (3/7) g3 q2 + (3/35) g2 t = R k + u q2 + w t
            const T u = T(-3.0 / 7.0) * g3, w = T(3.0 / 35.0) * g2;
            const T k = fma_(u, Rt, g4 * q3);
            A.S[0] = fma_(k, x, fma_(u, qx, fma_(w, bt[0], A.S[0])));
            A.S[1] = fma_(k, y, fma_(u, qy, fma_(w, bt[1], A.S[1])));
            A.S[2] = fma_(k, z, fma_(u, qz, fma_(w, bt[2], A.S[2])));
        }
    } else {
        A.L0 = fma_(m, g0, A.L0);
        A.L1[0] = fma_(-c1, x, A.L1[0]);
        A.L1[1] = fma_(-c1, y, A.L1[1]);
        A.L1[2] = fma_(-c1, z, A.L1[2]);
    }
    if (TGT_FULL) {
        const T s2 = m * g2;
        A.L2[0] = fma_(s2, xx, A.L2[0]);
        A.L2[1] = fma_(s2, xy, A.L2[1]);
        A.L2[2] = fma_(s2, xz, A.L2[2]);
        A.L2[3] = fma_(s2, yy, A.L2[3]);
        A.L2[4] = fma_(s2, yz, A.L2[4]);
        A.L2[5] = fma_(s2, zz, A.L2[5]);
        const T s3 = m * g3;
        const T tx3 = s3 * x, ty3 = s3 * y, tz3 = s3 * z;
        A.L3[0] = fma_(tx3, xx, A.L3[0]);
        A.L3[1] = fma_(tx3, xy, A.L3[1]);
        A.L3[2] = fma_(tx3, xz, A.L3[2]);
        A.L3[3] = fma_(tx3, yy, A.L3[3]);
        A.L3[4] = fma_(tx3, yz, A.L3[4]);
        A.L3[5] = fma_(tx3, zz, A.L3[5]);
        A.L3[6] = fma_(ty3, yy, A.L3[6]);
        A.L3[7] = fma_(ty3, yz, A.L3[7]);
        A.L3[8] = fma_(ty3, zz, A.L3[8]);
        A.L3[9] = fma_(tz3, zz, A.L3[9]);
        if (AM) {
            // A4 += m g4 R^4 (the target octupole is contracted once per
            // target): every quartic monomial is a square's multiple times a
            // quadratic one
            const T s4 = m * g4;
            const T txx = s4 * xx, tyy = s4 * yy, tzz = s4 * zz;
            A.A4[0] = fma_(txx, xx, A.A4[0]);
            A.A4[1] = fma_(txx, xy, A.A4[1]);
            A.A4[2] = fma_(txx, xz, A.A4[2]);
            A.A4[3] = fma_(txx, yy, A.A4[3]);
            A.A4[4] = fma_(txx, yz, A.A4[4]);
            A.A4[5] = fma_(txx, zz, A.A4[5]);
            A.A4[6] = fma_(tyy, xy, A.A4[6]);
            A.A4[7] = fma_(tyy, xz, A.A4[7]);
            A.A4[8] = fma_(tzz, xy, A.A4[8]);
            A.A4[9] = fma_(tzz, xz, A.A4[9]);
            A.A4[10] = fma_(tyy, yy, A.A4[10]);
            A.A4[11] = fma_(tyy, yz, A.A4[11]);
            A.A4[12] = fma_(tyy, zz, A.A4[12]);
            A.A4[13] = fma_(tzz, yz, A.A4[13]);
            A.A4[14] = fma_(tzz, zz, A.A4[14]);
        }
    }
}

// ---------------------------------------------------------------------------
// FP32-bulk form: the pair split by precision.  D is the FP64 scalar, F the
// FP32 one (a counting type on the host for the flop accounting; D = F =
// double in the host check of the split's algebra).
//
// In D: the monopole part of the pair, m_B D^(n)(R) for every order the
// target keeps (L0, L1; L2 and L3 at an interior target), and the
// correction's target sum A4 = sum m_B f4 R^4 -- everything that involves
// the source only through its mass -- from R formed in D; the per-pair value
// of the correction's source term S is added to a D sum.  In F: the
// contractions of the source's M2 and M3 with D^(n) (the quadrupole and
// octupole parts of L0 and L1, and S's per-pair value), from R and the radial
// factors formed again in F from the FP32 records; their L0/L1 parts are
// summed in F over at most a flush length of pairs and then added to the D
// sums (flush_split).
template <class D, class F> struct SplitAcc {
    D L0, L1[3];
    D L2[6], L3[10];  // until finish_split: sum m R R / r^5 and -sum m R R R / r^7
    D S[3];           // correction sum of the source octupoles
    D A4[15];         // sum m_B f4 R^4 of interior targets (order as in Acc),
                      // until finish_split sum m R^4 / r^9
    F l0, l1[3];      // partial sums of the source multipole parts of L0, L1
};

template <class D, class F> __host__ __device__ __forceinline__ void split_zero(SplitAcc<D, F>& A) {
    A.L0 = D(0.0);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        A.L1[i] = D(0.0);
        A.S[i] = D(0.0);
        A.l1[i] = F(0.0);
    }
    A.l0 = F(0.0);
#pragma unroll
    for (int i = 0; i < 6; i++) A.L2[i] = D(0.0);
#pragma unroll
    for (int i = 0; i < 10; i++) A.L3[i] = D(0.0);
#pragma unroll
    for (int i = 0; i < 15; i++) A.A4[i] = D(0.0);
}

// F -> D: exact widening for float (integer operations, common.cuh),
// identity for double.
__host__ __device__ __forceinline__ double to_d(double v) { return v; }
__host__ __device__ __forceinline__ double to_d(float v) { return widen(v); }

// Adds the F partial sums of L0 and L1 to the D sums and clears them.
template <class D, class F> __host__ __device__ __forceinline__ void flush_split(SplitAcc<D, F>& A) {
    A.L0 += to_d(A.l0);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        A.L1[i] += to_d(A.l1[i]);
        A.l1[i] = F(0.0);
    }
    A.l0 = F(0.0);
}

// Completes the D sums of an interior target once per item: the monopole
// sums are accumulated with the radial factors' constants left out (f2 =
// 3/r^5, f3 = -15/r^7 with the sign in the sum, f4 = 105/r^9), so they are
// multiplied in here; then the Kronecker parts of L2 and L3 from their traces
// (as finish_acc).
template <class D, class F> __host__ __device__ __forceinline__ void finish_split(SplitAcc<D, F>& A) {
#pragma unroll
    for (int i = 0; i < 6; i++) A.L2[i] = D(3.0) * A.L2[i];
#pragma unroll
    for (int i = 0; i < 10; i++) A.L3[i] = D(15.0) * A.L3[i];
#pragma unroll
    for (int i = 0; i < 15; i++) A.A4[i] = D(105.0) * A.A4[i];
    const D d1 = D(-1.0 / 3.0) * (A.L2[0] + A.L2[3] + A.L2[5]);
    const D Vx = D(-0.2) * (A.L3[0] + A.L3[3] + A.L3[5]);
    const D Vy = D(-0.2) * (A.L3[1] + A.L3[6] + A.L3[8]);
    const D Vz = D(-0.2) * (A.L3[2] + A.L3[7] + A.L3[9]);
    A.L2[0] += d1;
    A.L2[3] += d1;
    A.L2[5] += d1;
    A.L3[0] += D(3.0) * Vx;
    A.L3[1] += Vy;
    A.L3[2] += Vz;
    A.L3[3] += Vx;
    A.L3[5] += Vx;
    A.L3[6] += D(3.0) * Vy;
    A.L3[7] += Vz;
    A.L3[8] += Vy;
    A.L3[9] += D(3.0) * Vz;
}

// The correction's target term from the D sum A4 (as correction_target).
template <class D, class F>
__host__ __device__ __forceinline__ void correction_target_split(const SplitAcc<D, F>& S, const D* a,
                                                                 const D* t, D* P) {
    Acc<D> A;
#pragma unroll
    for (int i = 0; i < 15; i++) A.A4[i] = S.A4[i];
    correction_target(A, a, t, P);
}

// (x, y, z) = R' in D, (xf, yf, zf) = R' in F (from the FP32 records), m =
// source mass in D, b2/b3/bt = the source's M2', M3' and traces in F.
template <class D, class F, bool TGT_FULL, bool SRC_MULTI, bool AM>
__host__ __device__ __forceinline__ void m2l_pair_split(D x, D y, D z, D m, F xf, F yf, F zf,
                                                        const F* b2, const F* b3, const F* bt,
                                                        SplitAcc<D, F>& A) {
    // monopole part, D: w_k = m / r^(2k+1), so m f_k = (-1)^k (2k-1)!! w_k;
    // L1 and L3 take the sign (a negated FMA operand costs nothing), and
    // finish_split multiplies the L2, L3 and A4 sums by 3, 15 and 105
    const D r2 = fma_(x, x, fma_(y, y, z * z));
    const D f0 = rsqrt_(r2);
    const D ri2 = f0 * f0;
    const D w0 = m * f0;
    const D w1 = w0 * ri2;
    A.L0 += w0;
    A.L1[0] = fma_(-w1, x, A.L1[0]);
    A.L1[1] = fma_(-w1, y, A.L1[1]);
    A.L1[2] = fma_(-w1, z, A.L1[2]);
    if (TGT_FULL) {
        const D w2 = w1 * ri2;
        const D xx = x * x, yy = y * y, zz = z * z;
        const D xy = x * y, xz = x * z, yz = y * z;
        A.L2[0] = fma_(w2, xx, A.L2[0]);
        A.L2[1] = fma_(w2, xy, A.L2[1]);
        A.L2[2] = fma_(w2, xz, A.L2[2]);
        A.L2[3] = fma_(w2, yy, A.L2[3]);
        A.L2[4] = fma_(w2, yz, A.L2[4]);
        A.L2[5] = fma_(w2, zz, A.L2[5]);
        const D w3 = w2 * ri2;
        const D tx3 = w3 * x, ty3 = w3 * y, tz3 = w3 * z;
        A.L3[0] = fma_(-tx3, xx, A.L3[0]);
        A.L3[1] = fma_(-tx3, xy, A.L3[1]);
        A.L3[2] = fma_(-tx3, xz, A.L3[2]);
        A.L3[3] = fma_(-tx3, yy, A.L3[3]);
        A.L3[4] = fma_(-tx3, yz, A.L3[4]);
        A.L3[5] = fma_(-tx3, zz, A.L3[5]);
        A.L3[6] = fma_(-ty3, yy, A.L3[6]);
        A.L3[7] = fma_(-ty3, yz, A.L3[7]);
        A.L3[8] = fma_(-ty3, zz, A.L3[8]);
        A.L3[9] = fma_(-tz3, zz, A.L3[9]);
        if (AM) {
            const D w4 = w3 * ri2;
            const D txx = w4 * xx, tyy = w4 * yy, tzz = w4 * zz;
            A.A4[0] = fma_(txx, xx, A.A4[0]);
            A.A4[1] = fma_(txx, xy, A.A4[1]);
            A.A4[2] = fma_(txx, xz, A.A4[2]);
            A.A4[3] = fma_(txx, yy, A.A4[3]);
            A.A4[4] = fma_(txx, yz, A.A4[4]);
            A.A4[5] = fma_(txx, zz, A.A4[5]);
            A.A4[6] = fma_(tyy, xy, A.A4[6]);
            A.A4[7] = fma_(tyy, xz, A.A4[7]);
            A.A4[8] = fma_(tzz, xy, A.A4[8]);
            A.A4[9] = fma_(tzz, xz, A.A4[9]);
            A.A4[10] = fma_(tyy, yy, A.A4[10]);
            A.A4[11] = fma_(tyy, yz, A.A4[11]);
            A.A4[12] = fma_(tyy, zz, A.A4[12]);
            A.A4[13] = fma_(tzz, yz, A.A4[13]);
            A.A4[14] = fma_(tzz, zz, A.A4[14]);
        }
    }
    if (SRC_MULTI) {
        // source quadrupole and octupole parts, F
        const F r2f = fma_(xf, xf, fma_(yf, yf, zf * zf));
        const F g0 = rsqrt_(r2f);
        const F gi2 = g0 * g0;
        const F g1 = -(g0 * gi2);
        const F g2 = g1 * (F(-3.0) * gi2);
        const F g3 = g2 * (F(-5.0) * gi2);
        const F xx = xf * xf, yy = yf * yf, zz = zf * zf;
        const F xy2 = F(2.0) * (xf * yf), xz2 = F(2.0) * (xf * zf), yz2 = F(2.0) * (yf * zf);
        const F Mx = fma_(b2[0], xf, fma_(b2[1], yf, b2[2] * zf));
        const F My = fma_(b2[1], xf, fma_(b2[3], yf, b2[4] * zf));
        const F Mz = fma_(b2[2], xf, fma_(b2[4], yf, b2[5] * zf));
        const F xMx = fma_(xf, Mx, fma_(yf, My, zf * Mz));
        const F tr = bt[3];
        F qx, qy, qz;
        contract_rr(b3, xx, yy, zz, xy2, xz2, yz2, qx, qy, qz);
        const F q3 = fma_(xf, qx, fma_(yf, qy, zf * qz));
        const F Rt = fma_(xf, bt[0], fma_(yf, bt[1], zf * bt[2]));
        const F h2 = F(0.5) * g2;
        // L0 += (f2 xMx + f1 tr) / 2 - (f3 q3 + 3 f2 Rt) / 6
        A.l0 = fma_(F(0.5) * g1, tr, fma_(h2, xMx - Rt, fma_(F(-1.0 / 6.0) * g3, q3, A.l0)));
        // L1 += R (f3 xMx + f2 tr) / 2 + f2 M2 R
        const F e1 = fma_(F(0.5) * g3, xMx, h2 * tr);
        A.l1[0] = fma_(e1, xf, fma_(g2, Mx, A.l1[0]));
        A.l1[1] = fma_(e1, yf, fma_(g2, My, A.l1[1]));
        A.l1[2] = fma_(e1, zf, fma_(g2, Mz, A.l1[2]));
        if (AM) {
            // S += f4 R q3 + 3 f3 (q2 + R Rt) + 3 f2 t, each pair's value added to the D sum
            const F g4 = g3 * (F(-7.0) * gi2);
            const F u = F(3.0) * g3, w = F(3.0) * g2;
            const F k = fma_(u, Rt, g4 * q3);
            A.S[0] += to_d(fma_(k, xf, fma_(u, qx, w * bt[0])));
            A.S[1] += to_d(fma_(k, yf, fma_(u, qy, w * bt[1])));
            A.S[2] += to_d(fma_(k, zf, fma_(u, qz, w * bt[2])));
        }
    }
}

}  // namespace otfmm
