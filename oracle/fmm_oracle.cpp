// Oracle for the fast-multipole self-gravity solve on an octree of 8x8x8-cell
// subgrids (Octo-Tiger, arXiv 2412.15518, Sec. 4.3.1-4.3.2).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 CPU statement
// of what the GPU library computes.  Only the tests, the smoke check and the
// CPU-baseline leg of the benchmark may load it.  It shares no code, header,
// table or constant with the CUDA path.
//
// The paper states the method only in prose:
//   * gravity by a fast multipole method on the AMR octree (Sec. 2, Sec. 4.3.2);
//   * every tree node holds an 8x8x8 sub-grid of cells (Sec. 4.3.2);
//   * the FMM conserves linear momentum, and a special technique makes it
//     conserve angular momentum as well (Sec. 4.3.1);
//   * the GPU kernels walk a fixed stencil instead of an interaction list
//     (Sec. 5.5).
// Everything below that goes beyond those sentences is a reading written
// out step by step:
//   O0  a leaf cell is a point mass m = rho h^3 at its centre; free space;
//       phi(x) = -G sum m / |x - y|; the self pair is excluded.
//   U1  leaf moments: M0 = m, X = centre, M2 = M3 = 0 (moments about the COM,
//       so M1 = 0 identically).
//   U2  M2M: exact shift of children moments to the parent COM.
//   S   two level-L cells at integer offset d are near iff |d| <= 1/theta
//       (cell units).  A non-near pair is far at L = 0; at L >= 1 it is far
//       iff the parents are near.  Near pairs of two non-leaf cells descend.
//   F1  M2L of total order 3:  L^(n)_A += -G sum_{m<=3-n} (-1)^m/m!
//       M^(m)_B ._m D^(n+m)(X_A - X_B),  D^(k) = grad^k (1/r).
//   F2  angular-momentum correction (the top-order orbital force of the
//       truncated pair energy, applied uniformly to the target cell):
//       ac_A += -(G/6) D^(4)(R) ._3 [M3_B - (M0_B/M0_A) M3_A].
//   F3  a near pair with exactly one leaf cell interacts at its level by F1+F2.
//   N   a near pair of two leaf cells interacts exactly (point masses).
//   D1  L2L: exact shift of the degree-3 polynomial to the child; ac is
//       inherited.
//   D2  at a leaf cell: phi = L0 + near, g = -L1 + ac + near.
// All tensors are stored unpacked (3^n entries) so that every contraction is
// a plain index sum.  Sums run in a fixed order (target-major, sources in
// lexicographic (dz, dy, dx) order).  Built with -ffp-contract=off.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>
#include <omp.h>

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual number (value, derivative) so the same solve can be run
// for a directional derivative.
struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double a) : v(a), d(0) {}
    Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) {
    double s = std::sqrt(a.v);
    return Dual(s, a.d / (2.0 * s));
}
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
using std::sqrt;

template <class T> struct Mom {
    T m;
    T X[3];
    T M2[3][3];
    T M3[3][3][3];
};

template <class T> struct Loc {
    T L0;
    T L1[3];
    T L2[3][3];
    T L3[3][3][3];
    T ac[3];
};

template <class T> void zero_mom(Mom<T>& a) {
    a.m = T(0.0);
    for (int i = 0; i < 3; i++) {
        a.X[i] = T(0.0);
        for (int j = 0; j < 3; j++) {
            a.M2[i][j] = T(0.0);
            for (int k = 0; k < 3; k++) a.M3[i][j][k] = T(0.0);
        }
    }
}

template <class T> void zero_loc(Loc<T>& a) {
    a.L0 = T(0.0);
    for (int i = 0; i < 3; i++) {
        a.L1[i] = T(0.0);
        a.ac[i] = T(0.0);
        for (int j = 0; j < 3; j++) {
            a.L2[i][j] = T(0.0);
            for (int k = 0; k < 3; k++) a.L3[i][j][k] = T(0.0);
        }
    }
}

inline double kd(int i, int j) { return i == j ? 1.0 : 0.0; }

// D^(n)(R) = grad^n (1/|R|), n = 0..4, written from the closed form
//   D^(n) = sum over ways to pair indices by Kronecker deltas,
//   f_k = (-1)^k (2k-1)!! / r^(2k+1) multiplying the product of the
//   unpaired components R_i (k = n - #pairs).
template <class T> struct DTens {
    T D0;
    T D1[3];
    T D2[3][3];
    T D3[3][3][3];
    T D4[3][3][3][3];
};

template <class T> void dtensors(const T R[3], DTens<T>& D) {
    T r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    T r = sqrt(r2);
    T inv = T(1.0) / r;
    T inv2 = inv * inv;
    T f0 = inv;
    T f1 = T(-1.0) * f0 * inv2;
    T f2 = T(3.0) * f0 * inv2 * inv2;
    T f3 = T(-15.0) * f0 * inv2 * inv2 * inv2;
    T f4 = T(105.0) * f0 * inv2 * inv2 * inv2 * inv2;
    D.D0 = f0;
    for (int i = 0; i < 3; i++) {
        D.D1[i] = f1 * R[i];
        for (int j = 0; j < 3; j++) {
            D.D2[i][j] = f2 * R[i] * R[j] + f1 * kd(i, j);
            for (int k = 0; k < 3; k++) {
                D.D3[i][j][k] = f3 * R[i] * R[j] * R[k] +
                                f2 * (kd(i, j) * R[k] + kd(i, k) * R[j] + kd(j, k) * R[i]);
                for (int l = 0; l < 3; l++) {
                    D.D4[i][j][k][l] =
                        f4 * R[i] * R[j] * R[k] * R[l] +
                        f3 * (kd(i, j) * R[k] * R[l] + kd(i, k) * R[j] * R[l] +
                              kd(i, l) * R[j] * R[k] + kd(j, k) * R[i] * R[l] +
                              kd(j, l) * R[i] * R[k] + kd(k, l) * R[i] * R[j]) +
                        f2 * (kd(i, j) * kd(k, l) + kd(i, k) * kd(j, l) + kd(i, l) * kd(j, k));
                }
            }
        }
    }
}

// F1 + F2: contribution of source B to the expansion of target A.
template <class T>
void m2l(const Mom<T>& A, const Mom<T>& B, double G, int am, Loc<T>& out) {
    T R[3];
    for (int i = 0; i < 3; i++) R[i] = A.X[i] - B.X[i];
    DTens<T> D;
    dtensors(R, D);
    // n = 0: m = 0, 2, 3 (m = 1 vanishes about the COM)
    T s2 = T(0.0), s3 = T(0.0);
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++) {
            s2 += B.M2[j][k] * D.D2[j][k];
            for (int l = 0; l < 3; l++) s3 += B.M3[j][k][l] * D.D3[j][k][l];
        }
    out.L0 += T(-G) * (B.m * D.D0 + T(0.5) * s2 - T(1.0 / 6.0) * s3);
    // n = 1: m = 0, 2
    for (int i = 0; i < 3; i++) {
        T t = T(0.0);
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) t += B.M2[j][k] * D.D3[i][j][k];
        out.L1[i] += T(-G) * (B.m * D.D1[i] + T(0.5) * t);
    }
    // n = 2, 3: m = 0
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            out.L2[i][j] += T(-G) * B.m * D.D2[i][j];
            for (int k = 0; k < 3; k++) out.L3[i][j][k] += T(-G) * B.m * D.D3[i][j][k];
        }
    if (am) {
        // A cell of zero mass has M3 = 0 for non-negative densities; the
        // product of its undefined mass ratio and that zero tensor is taken as 0.
        T ratio = val(A.m) != 0.0 ? B.m / A.m : T(0.0);
        for (int i = 0; i < 3; i++) {
            T t = T(0.0);
            for (int j = 0; j < 3; j++)
                for (int k = 0; k < 3; k++)
                    for (int l = 0; l < 3; l++)
                        t += D.D4[i][j][k][l] * (B.M3[j][k][l] - ratio * A.M3[j][k][l]);
            out.ac[i] += T(-G / 6.0) * t;
        }
    }
}

// U2: moments of a parent from its children (exact shift to the parent COM).
// A parent of zero mass has no centre of mass; its moments are taken about
// `centre` (its geometric centre), or about the mean of the children's
// positions when no centre is given.
template <class T> void m2m(const Mom<T>* ch, int n, Mom<T>& P, const double* centre = nullptr) {
    zero_mom(P);
    for (int c = 0; c < n; c++) P.m += ch[c].m;
    for (int i = 0; i < 3; i++) {
        T s = T(0.0);
        if (val(P.m) != 0.0) {
            for (int c = 0; c < n; c++) s += ch[c].m * ch[c].X[i];
            P.X[i] = s / P.m;
        } else if (centre) {
            P.X[i] = T(centre[i]);
        } else {
            for (int c = 0; c < n; c++) s += ch[c].X[i];
            P.X[i] = s / T((double)n);
        }
    }
    for (int c = 0; c < n; c++) {
        T d[3];
        for (int i = 0; i < 3; i++) d[i] = ch[c].X[i] - P.X[i];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                P.M2[i][j] += ch[c].M2[i][j] + ch[c].m * d[i] * d[j];
                for (int k = 0; k < 3; k++)
                    P.M3[i][j][k] += ch[c].M3[i][j][k] + ch[c].M2[i][j] * d[k] +
                                     ch[c].M2[i][k] * d[j] + ch[c].M2[j][k] * d[i] +
                                     ch[c].m * d[i] * d[j] * d[k];
            }
    }
}

// D1: child expansion += exact shift of the parent's degree-3 polynomial by
// delta = X_child - X_parent; the correction acceleration is inherited.
template <class T> void l2l(const Loc<T>& P, const T d[3], Loc<T>& C) {
    T a0 = P.L0;
    for (int i = 0; i < 3; i++) {
        a0 += P.L1[i] * d[i];
        for (int j = 0; j < 3; j++) {
            a0 += T(0.5) * P.L2[i][j] * d[i] * d[j];
            for (int k = 0; k < 3; k++) a0 += T(1.0 / 6.0) * P.L3[i][j][k] * d[i] * d[j] * d[k];
        }
    }
    C.L0 += a0;
    for (int i = 0; i < 3; i++) {
        T a1 = P.L1[i];
        for (int j = 0; j < 3; j++) {
            a1 += P.L2[i][j] * d[j];
            for (int k = 0; k < 3; k++) a1 += T(0.5) * P.L3[i][j][k] * d[j] * d[k];
        }
        C.L1[i] += a1;
        for (int j = 0; j < 3; j++) {
            T a2 = P.L2[i][j];
            for (int k = 0; k < 3; k++) a2 += P.L3[i][j][k] * d[k];
            C.L2[i][j] += a2;
            for (int k = 0; k < 3; k++) C.L3[i][j][k] += P.L3[i][j][k];
        }
        C.ac[i] += P.ac[i];
    }
}

// ---------------------------------------------------------------------------
// Octree of 8^3-cell nodes (O1).  A level-L node (x, y, z) covers the cube
// [x, x+1) * size / 2^L (per axis) and holds cells [8x, 8x+8) at level L.
struct Node {
    int x, y, z;
    int leaf_id;  // caller's leaf index, or -1 for an interior node
};

inline uint64_t key3(int x, int y, int z) {
    return (uint64_t)(uint32_t)x | ((uint64_t)(uint32_t)y << 21) | ((uint64_t)(uint32_t)z << 42);
}

struct Tree {
    int Lmax = -1;
    double origin[3] = {0, 0, 0};
    double size = 1.0;
    std::vector<std::vector<Node>> lev;
    std::vector<std::unordered_map<uint64_t, int>> map;

    int find(int L, int x, int y, int z) const {
        if (L < 0 || L > Lmax) return -1;
        int n = 1 << L;
        if (x < 0 || y < 0 || z < 0 || x >= n || y >= n || z >= n) return -1;
        auto it = map[L].find(key3(x, y, z));
        return it == map[L].end() ? -1 : it->second;
    }
    double h(int L) const { return size / (8.0 * (double)(1 << L)); }
    // index of cell (cx, cy, cz) at level L in that level's cell array, or -1
    long cell(int L, int cx, int cy, int cz) const {
        int nd = find(L, cx >> 3, cy >> 3, cz >> 3);
        if (cx < 0 || cy < 0 || cz < 0) return -1;
        if (nd < 0) return -1;
        return (long)nd * 512 + (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7);
    }
};

enum { ORC_OK = 0, ORC_BAD_LEAF = -1, ORC_OVERLAP = -2, ORC_INCOMPLETE = -3 };

int build_tree(int n_leaf, const int32_t* leaves, const double* origin, double size, Tree& t) {
    t = Tree();
    if (origin)
        for (int i = 0; i < 3; i++) t.origin[i] = origin[i];
    t.size = size;
    int Lmax = 0;
    for (int i = 0; i < n_leaf; i++) {
        int L = leaves[4 * i];
        if (L < 0 || L > 20) return ORC_BAD_LEAF;
        for (int a = 1; a < 4; a++)
            if (leaves[4 * i + a] < 0 || leaves[4 * i + a] >= (1 << L)) return ORC_BAD_LEAF;
        if (L > Lmax) Lmax = L;
    }
    if (n_leaf <= 0) return ORC_BAD_LEAF;
    t.Lmax = Lmax;
    t.lev.assign(Lmax + 1, {});
    t.map.assign(Lmax + 1, {});
    for (int i = 0; i < n_leaf; i++) {
        int L = leaves[4 * i], x = leaves[4 * i + 1], y = leaves[4 * i + 2], z = leaves[4 * i + 3];
        auto it = t.map[L].find(key3(x, y, z));
        if (it != t.map[L].end()) return ORC_OVERLAP;  // duplicate, or a leaf inside a leaf
        t.map[L][key3(x, y, z)] = (int)t.lev[L].size();
        t.lev[L].push_back({x, y, z, i});
    }
    // ancestors
    for (int i = 0; i < n_leaf; i++) {
        int L = leaves[4 * i], x = leaves[4 * i + 1], y = leaves[4 * i + 2], z = leaves[4 * i + 3];
        for (int l = L - 1; l >= 0; l--) {
            x >>= 1; y >>= 1; z >>= 1;
            auto it = t.map[l].find(key3(x, y, z));
            if (it != t.map[l].end()) {
                if (t.lev[l][it->second].leaf_id >= 0) return ORC_OVERLAP;
                break;  // this ancestor and its own ancestors already exist
            }
            t.map[l][key3(x, y, z)] = (int)t.lev[l].size();
            t.lev[l].push_back({x, y, z, -1});
        }
    }
    // completeness: every interior node has all eight children
    for (int l = 0; l < Lmax; l++)
        for (const Node& nd : t.lev[l]) {
            if (nd.leaf_id >= 0) continue;
            for (int c = 0; c < 8; c++)
                if (t.find(l + 1, 2 * nd.x + (c & 1), 2 * nd.y + ((c >> 1) & 1),
                           2 * nd.z + ((c >> 2) & 1)) < 0)
                    return ORC_INCOMPLETE;
        }
    if (t.lev[0].size() != 1) return ORC_INCOMPLETE;
    return ORC_OK;
}

inline int local_of(int i, int j, int k) { return i + 8 * j + 64 * k; }

// ---------------------------------------------------------------------------
// The solve, templated on the scalar type (double, or Dual for a
// directional derivative).
template <class T> struct Work {
    std::vector<std::vector<Mom<T>>> mom;  // per level, per cell
    std::vector<std::vector<Loc<T>>> loc;
    std::vector<std::vector<T>> nphi;      // near-field potential (leaf cells)
    std::vector<std::vector<T>> ng;        // near-field acceleration, 3 per cell
    std::vector<std::vector<char>> need;   // cells whose expansion is required
    int64_t n_m2l = 0, n_p2p = 0, n_seam = 0;
};

template <class T> void upward(const Tree& t, const T* rho, Work<T>& w) {
    w.mom.assign(t.Lmax + 1, {});
    for (int L = t.Lmax; L >= 0; L--) {
        const auto& nodes = t.lev[L];
        w.mom[L].resize(nodes.size() * 512);
        double h = t.h(L);
#pragma omp parallel for schedule(static)
        for (long n = 0; n < (long)nodes.size(); n++) {
            const Node& nd = nodes[n];
            for (int k = 0; k < 8; k++)
                for (int j = 0; j < 8; j++)
                    for (int i = 0; i < 8; i++) {
                        Mom<T>& M = w.mom[L][n * 512 + local_of(i, j, k)];
                        int cx = 8 * nd.x + i, cy = 8 * nd.y + j, cz = 8 * nd.z + k;
                        if (nd.leaf_id >= 0) {
                            // U1: point mass at the cell centre
                            zero_mom(M);
                            M.m = rho[(long)nd.leaf_id * 512 + local_of(i, j, k)] * T(h * h * h);
                            M.X[0] = T(t.origin[0] + (cx + 0.5) * h);
                            M.X[1] = T(t.origin[1] + (cy + 0.5) * h);
                            M.X[2] = T(t.origin[2] + (cz + 0.5) * h);
                        } else {
                            Mom<T> ch[8];
                            for (int c = 0; c < 8; c++) {
                                long ci = t.cell(L + 1, 2 * cx + (c & 1), 2 * cy + ((c >> 1) & 1),
                                                 2 * cz + ((c >> 2) & 1));
                                ch[c] = w.mom[L + 1][ci];
                            }
                            const double ctr[3] = {t.origin[0] + (cx + 0.5) * h,
                                                   t.origin[1] + (cy + 0.5) * h,
                                                   t.origin[2] + (cz + 0.5) * h};
                            m2m(ch, 8, M, ctr);
                        }
                    }
        }
    }
}

// S: the interaction rules for two level-L cells a, b (global cell indices).
// Returns 0 = none, 1 = far (M2L), 2 = near leaf pair (exact), 3 = near
// mixed pair (F3, M2L), 4 = near pair of two interior cells (descends).
inline int classify(int L, const int a[3], const int b[3], double inv_theta2, bool leaf_a,
                    bool leaf_b) {
    double d2 = 0.0;
    for (int i = 0; i < 3; i++) d2 += (double)(a[i] - b[i]) * (double)(a[i] - b[i]);
    bool near = d2 <= inv_theta2;
    if (near) {
        if (leaf_a && leaf_b) return 2;
        if (leaf_a || leaf_b) return 3;
        return 4;
    }
    if (L == 0) return 1;
    double p2 = 0.0;
    for (int i = 0; i < 3; i++) {
        double dp = (double)((a[i] >> 1) - (b[i] >> 1));
        p2 += dp * dp;
    }
    return p2 <= inv_theta2 ? 1 : 0;
}

// Largest |d_i| at which two cells at L >= 1 can still have near parents:
// parents at offset D with |D_i| <= floor(1/theta) have children at most
// 2 floor(1/theta) + 1 apart.
inline int window(double theta) { return 2 * (int)std::floor(1.0 / theta + 1e-12) + 1; }

template <class T>
void interactions(const Tree& t, double theta, double G, int am, Work<T>& w, bool count) {
    double it2 = 1.0 / (theta * theta);
    int W = window(theta);
    w.loc.assign(t.Lmax + 1, {});
    w.nphi.assign(t.Lmax + 1, {});
    w.ng.assign(t.Lmax + 1, {});
    int64_t c_m2l = 0, c_p2p = 0, c_seam = 0;
    for (int L = 0; L <= t.Lmax; L++) {
        const auto& nodes = t.lev[L];
        long nc = (long)nodes.size() * 512;
        w.loc[L].resize(nc);
        w.nphi[L].assign(nc, T(0.0));
        w.ng[L].assign(3 * nc, T(0.0));
        int ncell = 8 << L;
        int lo_w = (L == 0) ? ncell : W;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : c_m2l, c_p2p, c_seam)
        for (long ci = 0; ci < nc; ci++) {
            Loc<T>& out = w.loc[L][ci];
            zero_loc(out);
            if (!w.need[L][ci]) continue;
            const Node& nd = nodes[ci / 512];
            int l = (int)(ci % 512);
            int a[3] = {8 * nd.x + (l & 7), 8 * nd.y + ((l >> 3) & 7), 8 * nd.z + (l >> 6)};
            bool leaf_a = nd.leaf_id >= 0;
            const Mom<T>& A = w.mom[L][ci];
            T phi_n = T(0.0), gn[3] = {T(0.0), T(0.0), T(0.0)};
            int lo[3], hi[3];
            for (int i = 0; i < 3; i++) {
                lo[i] = a[i] - lo_w < 0 ? 0 : a[i] - lo_w;
                hi[i] = a[i] + lo_w > ncell - 1 ? ncell - 1 : a[i] + lo_w;
            }
            for (int bz = lo[2]; bz <= hi[2]; bz++)
                for (int by = lo[1]; by <= hi[1]; by++)
                    for (int bx = lo[0]; bx <= hi[0]; bx++) {
                        int b[3] = {bx, by, bz};
                        if (bx == a[0] && by == a[1] && bz == a[2]) continue;  // self pair excluded
                        int bn = t.find(L, b[0] >> 3, b[1] >> 3, b[2] >> 3);
                        if (bn < 0) continue;  // that region is covered by a coarser leaf
                        bool leaf_b = nodes[bn].leaf_id >= 0;
                        int cls = classify(L, a, b, it2, leaf_a, leaf_b);
                        if (cls == 0 || cls == 4) continue;
                        const Mom<T>& B = w.mom[L][(long)bn * 512 +
                                                   local_of(b[0] & 7, b[1] & 7, b[2] & 7)];
                        if (cls == 2) {
                            // N: exact point-mass interaction
                            T r[3];
                            for (int i = 0; i < 3; i++) r[i] = A.X[i] - B.X[i];
                            T rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                            T ir = T(1.0) / rr;
                            phi_n += T(-G) * B.m * ir;
                            T ir3 = ir * ir * ir;
                            for (int i = 0; i < 3; i++) gn[i] += T(-G) * B.m * r[i] * ir3;
                            c_p2p++;
                        } else {
                            m2l(A, B, G, am, out);
                            if (cls == 1) c_m2l++;
                            else c_seam++;
                        }
                    }
            w.nphi[L][ci] = phi_n;
            for (int i = 0; i < 3; i++) w.ng[L][3 * ci + i] = gn[i];
        }
    }
    if (count) {
        w.n_m2l = c_m2l;
        w.n_p2p = c_p2p;
        w.n_seam = c_seam;
    }
}

template <class T> void downward(const Tree& t, Work<T>& w) {
    for (int L = 1; L <= t.Lmax; L++) {
        const auto& nodes = t.lev[L];
        long nc = (long)nodes.size() * 512;
#pragma omp parallel for schedule(static)
        for (long ci = 0; ci < nc; ci++) {
            if (!w.need[L][ci]) continue;
            const Node& nd = nodes[ci / 512];
            int l = (int)(ci % 512);
            int a[3] = {8 * nd.x + (l & 7), 8 * nd.y + ((l >> 3) & 7), 8 * nd.z + (l >> 6)};
            long pi = t.cell(L - 1, a[0] >> 1, a[1] >> 1, a[2] >> 1);
            T d[3];
            for (int i = 0; i < 3; i++) d[i] = w.mom[L][ci].X[i] - w.mom[L - 1][pi].X[i];
            l2l(w.loc[L - 1][pi], d, w.loc[L][ci]);
        }
    }
}

// Self potential of a uniform cube of side 1 and density 1 at its centre:
//   C = int_{[-1/2,1/2]^3} dV / |r|.
// By the 48-fold symmetry the cube splits into 3 pyramids per octant with
// apex at the centre; in the pyramid where x is the largest coordinate,
// substituting y = x u, z = x v gives int_0^{1/2} x dx * I = I / 8 with
// I = int_0^1 int_0^1 du dv / sqrt(1 + u^2 + v^2), hence C = 8 * 3 * I / 8 = 3 I.
// I is evaluated by tensor-product Gauss-Legendre quadrature (smooth
// integrand), nodes found by Newton iteration on P_n.
double cube_self_constant() {
    const int n = 48;
    double I = 0.0;
    std::vector<double> x(n), wt(n);
    for (int i = 0; i < n; i++) {
        // i-th root of the Legendre polynomial P_n by Newton's method
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);  // P_n'(z)
            double step = p1 / dp;
            z -= step;
            if (std::fabs(step) < 1e-15) break;
        }
        // weight on [-1, 1] is 2 / ((1 - z^2) P_n'(z)^2); mapped to [0, 1] it halves
        x[i] = 0.5 * (z + 1.0);
        wt[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) I += wt[i] * wt[j] / std::sqrt(1.0 + x[i] * x[i] + x[j] * x[j]);
    return 3.0 * I;
}

template <class T>
void evaluate(const Tree& t, const T* rho, double G, int self_term, Work<T>& w, T* phi, T* g,
              const int64_t* sample, long n_sample) {
    double C = self_term ? cube_self_constant() : 0.0;
    std::unordered_map<long, std::vector<long>> slots;
    if (sample)
        for (long s = 0; s < n_sample; s++) slots[sample[s]].push_back(s);
    for (int L = 0; L <= t.Lmax; L++) {
        const auto& nodes = t.lev[L];
        double h = t.h(L);
        for (long n = 0; n < (long)nodes.size(); n++) {
            const Node& nd = nodes[n];
            if (nd.leaf_id < 0) continue;
            for (int l = 0; l < 512; l++) {
                long ci = n * 512 + l;
                if (!w.need[L][ci]) continue;
                long out = (long)nd.leaf_id * 512 + l;
                const Loc<T>& E = w.loc[L][ci];
                T p = E.L0 + w.nphi[L][ci];
                if (self_term) p += T(-G * h * h * C) * rho[out];
                T gg[3];
                for (int i = 0; i < 3; i++) gg[i] = T(-1.0) * E.L1[i] + E.ac[i] + w.ng[L][3 * ci + i];
                if (sample) {
                    // write into the sample slot(s) that ask for this cell
                    auto it = slots.find(out);
                    if (it == slots.end()) continue;
                    for (long s : it->second) {
                        phi[s] = p;
                        for (int i = 0; i < 3; i++) g[3 * s + i] = gg[i];
                    }
                } else {
                    phi[out] = p;
                    for (int i = 0; i < 3; i++) g[((long)nd.leaf_id * 3 + i) * 512 + l] = gg[i];
                }
            }
        }
    }
}

// Mark which cells need an expansion: all cells (full solve) or the sampled
// leaf cells and their ancestors.
template <class T>
void mark_need(const Tree& t, Work<T>& w, const int64_t* sample, long n_sample,
               const std::vector<std::pair<int, long>>& leaf_cell_of) {
    w.need.assign(t.Lmax + 1, {});
    for (int L = 0; L <= t.Lmax; L++) w.need[L].assign(t.lev[L].size() * 512, sample ? 0 : 1);
    if (!sample) return;
    for (long s = 0; s < n_sample; s++) {
        long leaf = sample[s] / 512;
        int l = (int)(sample[s] % 512);
        int L = leaf_cell_of[leaf].first;
        long ci = leaf_cell_of[leaf].second * 512 + l;
        const Node& nd = t.lev[L][ci / 512];
        int a[3] = {8 * nd.x + (l & 7), 8 * nd.y + ((l >> 3) & 7), 8 * nd.z + (l >> 6)};
        for (int q = L; q >= 0; q--) {
            long cq = t.cell(q, a[0] >> (L - q), a[1] >> (L - q), a[2] >> (L - q));
            w.need[q][cq] = 1;
        }
    }
}

template <class T>
int solve(const Tree& t, const T* rho, double theta, double G, int am, int self_term, T* phi, T* g,
          const int64_t* sample, long n_sample, int64_t* counts) {
    std::vector<std::pair<int, long>> leaf_cell_of;
    long n_leaf = 0;
    for (int L = 0; L <= t.Lmax; L++)
        for (const Node& nd : t.lev[L])
            if (nd.leaf_id >= 0) n_leaf++;
    leaf_cell_of.resize(n_leaf);
    for (int L = 0; L <= t.Lmax; L++)
        for (long n = 0; n < (long)t.lev[L].size(); n++)
            if (t.lev[L][n].leaf_id >= 0) leaf_cell_of[t.lev[L][n].leaf_id] = {L, n};
    if (sample)
        for (long s = 0; s < n_sample; s++)
            if (sample[s] < 0 || sample[s] >= n_leaf * 512) return ORC_BAD_LEAF;
    Work<T> w;
    mark_need(t, w, sample, n_sample, leaf_cell_of);
    upward(t, rho, w);
    interactions(t, theta, G, am, w, counts != nullptr);
    downward(t, w);
    evaluate(t, rho, G, self_term, w, phi, g, sample, n_sample);
    if (counts) {
        counts[0] = w.n_m2l;
        counts[1] = w.n_p2p;
        counts[2] = w.n_seam;
    }
    return ORC_OK;
}

// ---------------------------------------------------------------------------
// Adjoint (reverse sweep) of the solve, FP64, full unpacked tensors.
// J = sum_c (w1_c phi_c + w2_c . g_c); every step above is reversed in the
// opposite order with the chain rule written out entry by entry.

// D^(5)_{ijklm}: next term of the same closed form: f5 RRRRR + f4 (10 terms
// delta RRR) + f3 (15 terms delta delta R), f5 = -945 / r^11.
void dtensor5(const double R[3], double D5[3][3][3][3][3]) {
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    double r = std::sqrt(r2);
    double inv = 1.0 / r, inv2 = inv * inv;
    double f3 = -15.0 * inv * inv2 * inv2 * inv2;
    double f4 = 105.0 * inv * inv2 * inv2 * inv2 * inv2;
    double f5 = -945.0 * inv * inv2 * inv2 * inv2 * inv2 * inv2;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++)
                    for (int m = 0; m < 3; m++) {
                        double v = f5 * R[i] * R[j] * R[k] * R[l] * R[m];
                        v += f4 * (kd(i, j) * R[k] * R[l] * R[m] + kd(i, k) * R[j] * R[l] * R[m] +
                                   kd(i, l) * R[j] * R[k] * R[m] + kd(i, m) * R[j] * R[k] * R[l] +
                                   kd(j, k) * R[i] * R[l] * R[m] + kd(j, l) * R[i] * R[k] * R[m] +
                                   kd(j, m) * R[i] * R[k] * R[l] + kd(k, l) * R[i] * R[j] * R[m] +
                                   kd(k, m) * R[i] * R[j] * R[l] + kd(l, m) * R[i] * R[j] * R[k]);
                        v += f3 * (kd(i, j) * (kd(k, l) * R[m] + kd(k, m) * R[l] + kd(l, m) * R[k]) +
                                   kd(i, k) * (kd(j, l) * R[m] + kd(j, m) * R[l] + kd(l, m) * R[j]) +
                                   kd(i, l) * (kd(j, k) * R[m] + kd(j, m) * R[k] + kd(k, m) * R[j]) +
                                   kd(i, m) * (kd(j, k) * R[l] + kd(j, l) * R[k] + kd(k, l) * R[j]) +
                                   kd(j, k) * kd(l, m) * R[i] + kd(j, l) * kd(k, m) * R[i] +
                                   kd(j, m) * kd(k, l) * R[i]);
                        D5[i][j][k][l][m] = v;
                    }
}

struct MomBar {
    double m, X[3], M2[3][3], M3[3][3][3];
};

void zero_bar(MomBar& b) { std::memset(&b, 0, sizeof(b)); }
void zero_locd(Loc<double>& a) { zero_loc(a); }

// Reverse of m2l(A, B) given the adjoint E of the target expansion: adds the
// adjoints of A's and/or B's moments (and positions).  as_target / as_source
// select which side is accumulated (the pair is visited once from each side).
void m2l_reverse(const Mom<double>& A, const Mom<double>& B, double G, int am,
                 const Loc<double>& E, MomBar* bA, MomBar* bB, bool need_R) {
    double R[3];
    for (int i = 0; i < 3; i++) R[i] = A.X[i] - B.X[i];
    DTens<double> D;
    dtensors(R, D);
    static thread_local double D5[3][3][3][3][3];
    if (need_R && am) dtensor5(R, D5);
    // adjoints of the D tensors
    double b0, b1[3], b2[3][3], b3[3][3][3], b4[3][3][3][3];
    b0 = -G * E.L0 * B.m;
    for (int i = 0; i < 3; i++) b1[i] = -G * E.L1[i] * B.m;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            b2[i][j] = -G * (0.5 * E.L0 * B.M2[i][j] + E.L2[i][j] * B.m);
            for (int k = 0; k < 3; k++)
                b3[i][j][k] = -G * (-(1.0 / 6.0) * E.L0 * B.M3[i][j][k] +
                                    0.5 * E.L1[i] * B.M2[j][k] + E.L3[i][j][k] * B.m);
        }
    // zero-mass target: ratio term taken as 0 (and not differentiated)
    const bool live_A = A.m != 0.0;
    double ratio = live_A ? B.m / A.m : 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++)
                    b4[i][j][k][l] =
                        am ? -(G / 6.0) * E.ac[i] * (B.M3[j][k][l] - ratio * A.M3[j][k][l]) : 0.0;
    // R adjoint: sum_n bn . D^(n+1) (only needed when the side whose position
    // adjoint is accumulated is an interior cell; leaf positions are constants)
    double Rb[3] = {0.0, 0.0, 0.0};
    for (int p = 0; p < 3 && need_R; p++) {
        double v = b0 * D.D1[p];
        for (int i = 0; i < 3; i++) {
            v += b1[i] * D.D2[i][p];
            for (int j = 0; j < 3; j++) {
                v += b2[i][j] * D.D3[i][j][p];
                for (int k = 0; k < 3; k++) {
                    v += b3[i][j][k] * D.D4[i][j][k][p];
                    if (am)
                        for (int l = 0; l < 3; l++) v += b4[i][j][k][l] * D5[i][j][k][l][p];
                }
            }
        }
        Rb[p] = v;
    }
    if (bA) {
        for (int p = 0; p < 3; p++) bA->X[p] += Rb[p];
        if (am) {
            // ac depends on A through -(m_B / m_A) M3_A
            double s = 0.0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++)
                    for (int k = 0; k < 3; k++)
                        for (int l = 0; l < 3; l++) {
                            double t = -(G / 6.0) * E.ac[i] * D.D4[i][j][k][l];
                            bA->M3[j][k][l] += t * (-ratio);
                            s += t * A.M3[j][k][l];
                        }
            if (live_A) bA->m += s * (B.m / (A.m * A.m));
        }
    }
    if (bB) {
        for (int p = 0; p < 3; p++) bB->X[p] -= Rb[p];
        double mb = E.L0 * D.D0;
        for (int i = 0; i < 3; i++) {
            mb += E.L1[i] * D.D1[i];
            for (int j = 0; j < 3; j++) {
                mb += E.L2[i][j] * D.D2[i][j];
                for (int k = 0; k < 3; k++) mb += E.L3[i][j][k] * D.D3[i][j][k];
            }
        }
        bB->m += -G * mb;
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) {
                double t = 0.5 * E.L0 * D.D2[j][k];
                for (int i = 0; i < 3; i++) t += 0.5 * E.L1[i] * D.D3[i][j][k];
                bB->M2[j][k] += -G * t;
                for (int l = 0; l < 3; l++) bB->M3[j][k][l] += -G * (-(1.0 / 6.0)) * E.L0 * D.D3[j][k][l];
            }
        if (am) {
            double s = 0.0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++)
                    for (int k = 0; k < 3; k++)
                        for (int l = 0; l < 3; l++) {
                            double t = -(G / 6.0) * E.ac[i] * D.D4[i][j][k][l];
                            bB->M3[j][k][l] += t;
                            s += t * A.M3[j][k][l];
                        }
            if (live_A) bB->m += s * (-1.0 / A.m);
        }
    }
}

// Reverse of l2l(P, d, C) given the child adjoint Cb: adds into the parent
// adjoint Pb and returns the adjoint of d.
void l2l_reverse(const Loc<double>& P, const double d[3], const Loc<double>& Cb, Loc<double>& Pb,
                 double db[3]) {
    Pb.L0 += Cb.L0;
    for (int i = 0; i < 3; i++) {
        Pb.L1[i] += Cb.L0 * d[i] + Cb.L1[i];
        Pb.ac[i] += Cb.ac[i];
        for (int j = 0; j < 3; j++) {
            Pb.L2[i][j] += 0.5 * Cb.L0 * d[i] * d[j] + Cb.L1[i] * d[j] + Cb.L2[i][j];
            for (int k = 0; k < 3; k++)
                Pb.L3[i][j][k] += (1.0 / 6.0) * Cb.L0 * d[i] * d[j] * d[k] +
                                  0.5 * Cb.L1[i] * d[j] * d[k] + Cb.L2[i][j] * d[k] + Cb.L3[i][j][k];
        }
    }
    for (int p = 0; p < 3; p++) {
        double a0 = P.L1[p];
        for (int j = 0; j < 3; j++) {
            a0 += 0.5 * (P.L2[p][j] + P.L2[j][p]) * d[j];
            for (int k = 0; k < 3; k++)
                a0 += (1.0 / 6.0) * (P.L3[p][j][k] + P.L3[j][p][k] + P.L3[j][k][p]) * d[j] * d[k];
        }
        double v = Cb.L0 * a0;
        for (int i = 0; i < 3; i++) {
            double a1 = P.L2[i][p];
            for (int k = 0; k < 3; k++) a1 += 0.5 * (P.L3[i][p][k] + P.L3[i][k][p]) * d[k];
            v += Cb.L1[i] * a1;
            for (int j = 0; j < 3; j++) v += Cb.L2[i][j] * P.L3[i][j][p];
        }
        db[p] = v;
    }
}

// Reverse of m2m(ch, 8, P) given the parent adjoint Pb (its X entry is the
// total adjoint of the parent's centre of mass from all other uses): adds
// into the children's adjoints.
void m2m_reverse(const Mom<double>* ch, int n, const Mom<double>& P, const MomBar& Pb,
                 MomBar* cb) {
    double Xb[3] = {Pb.X[0], Pb.X[1], Pb.X[2]};
    for (int c = 0; c < n; c++) {
        double d[3];
        for (int i = 0; i < 3; i++) d[i] = ch[c].X[i] - P.X[i];
        double dbar[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double t2 = Pb.M2[i][j];
                cb[c].M2[i][j] += t2;
                cb[c].m += t2 * d[i] * d[j];
                dbar[i] += t2 * ch[c].m * d[j];
                dbar[j] += t2 * ch[c].m * d[i];
                for (int k = 0; k < 3; k++) {
                    double t3 = Pb.M3[i][j][k];
                    cb[c].M3[i][j][k] += t3;
                    cb[c].M2[i][j] += t3 * d[k];
                    cb[c].M2[i][k] += t3 * d[j];
                    cb[c].M2[j][k] += t3 * d[i];
                    dbar[k] += t3 * ch[c].M2[i][j];
                    dbar[j] += t3 * ch[c].M2[i][k];
                    dbar[i] += t3 * ch[c].M2[j][k];
                    cb[c].m += t3 * d[i] * d[j] * d[k];
                    dbar[i] += t3 * ch[c].m * d[j] * d[k];
                    dbar[j] += t3 * ch[c].m * d[i] * d[k];
                    dbar[k] += t3 * ch[c].m * d[i] * d[j];
                }
            }
        for (int i = 0; i < 3; i++) {
            cb[c].X[i] += dbar[i];
            Xb[i] -= dbar[i];
        }
    }
    // X_P = sum m_k X_k / M,  M = sum m_k (a constant centre when M = 0)
    for (int c = 0; c < n; c++) {
        double s = 0.0;
        for (int i = 0; i < 3 && P.m != 0.0; i++) {
            cb[c].X[i] += Xb[i] * ch[c].m / P.m;
            s += Xb[i] * (ch[c].X[i] - P.X[i]) / P.m;
        }
        cb[c].m += s + Pb.m;
    }
}

int gradient(const Tree& t, const double* rho, double theta, double G, int am, int self_term,
             const double* w1, const double* w2, double* drho) {
    long n_leaf = 0;
    for (int L = 0; L <= t.Lmax; L++)
        for (const Node& nd : t.lev[L]) n_leaf += nd.leaf_id >= 0;
    std::vector<std::pair<int, long>> leaf_cell_of(n_leaf);
    for (int L = 0; L <= t.Lmax; L++)
        for (long n = 0; n < (long)t.lev[L].size(); n++)
            if (t.lev[L][n].leaf_id >= 0) leaf_cell_of[t.lev[L][n].leaf_id] = {L, n};
    Work<double> w;
    mark_need(t, w, nullptr, 0, leaf_cell_of);
    upward(t, rho, w);
    interactions(t, theta, G, am, w, false);
    downward(t, w);
    // adjoints of the expansions: seeds at leaf cells
    std::vector<std::vector<Loc<double>>> Eb(t.Lmax + 1);
    std::vector<std::vector<MomBar>> Mb(t.Lmax + 1);
    for (int L = 0; L <= t.Lmax; L++) {
        long nc = (long)t.lev[L].size() * 512;
        Eb[L].resize(nc);
        Mb[L].resize(nc);
        for (long ci = 0; ci < nc; ci++) {
            zero_loc(Eb[L][ci]);
            zero_bar(Mb[L][ci]);
        }
        for (long n = 0; n < (long)t.lev[L].size(); n++) {
            int leaf = t.lev[L][n].leaf_id;
            if (leaf < 0) continue;
            for (int l = 0; l < 512; l++) {
                Loc<double>& e = Eb[L][n * 512 + l];
                e.L0 = w1[(long)leaf * 512 + l];
                for (int i = 0; i < 3; i++) {
                    double wg = w2[((long)leaf * 3 + i) * 512 + l];
                    e.L1[i] = -wg;
                    e.ac[i] = wg;
                }
            }
        }
    }
    // L2L reverse, bottom-up, gathered at each parent
    for (int L = t.Lmax; L >= 1; L--) {
        const auto& pn = t.lev[L - 1];
        long np = (long)pn.size() * 512;
#pragma omp parallel for schedule(static)
        for (long pi = 0; pi < np; pi++) {
            const Node& nd = pn[pi / 512];
            if (nd.leaf_id >= 0) continue;
            int l = (int)(pi % 512);
            int a[3] = {8 * nd.x + (l & 7), 8 * nd.y + ((l >> 3) & 7), 8 * nd.z + (l >> 6)};
            for (int c = 0; c < 8; c++) {
                long ci = t.cell(L, 2 * a[0] + (c & 1), 2 * a[1] + ((c >> 1) & 1), 2 * a[2] + (c >> 2));
                double d[3], db[3];
                for (int i = 0; i < 3; i++) d[i] = w.mom[L][ci].X[i] - w.mom[L - 1][pi].X[i];
                l2l_reverse(w.loc[L - 1][pi], d, Eb[L][ci], Eb[L - 1][pi], db);
                for (int i = 0; i < 3; i++) {
                    Mb[L][ci].X[i] += db[i];
                    Mb[L - 1][pi].X[i] -= db[i];
                }
            }
        }
    }
    // M2L and near-pair reverse, gathered per cell over both of its roles
    double it2 = 1.0 / (theta * theta);
    int W = window(theta);
    for (int L = 0; L <= t.Lmax; L++) {
        const auto& nodes = t.lev[L];
        long nc = (long)nodes.size() * 512;
        int ncell = 8 << L;
        int lo_w = (L == 0) ? ncell : W;
#pragma omp parallel for schedule(dynamic, 1)
        for (long ci = 0; ci < nc; ci++) {
            const Node& nd = nodes[ci / 512];
            int l = (int)(ci % 512);
            int a[3] = {8 * nd.x + (l & 7), 8 * nd.y + ((l >> 3) & 7), 8 * nd.z + (l >> 6)};
            bool leaf_a = nd.leaf_id >= 0;
            const Mom<double>& C = w.mom[L][ci];
            int lo[3], hi[3];
            for (int i = 0; i < 3; i++) {
                lo[i] = a[i] - lo_w < 0 ? 0 : a[i] - lo_w;
                hi[i] = a[i] + lo_w > ncell - 1 ? ncell - 1 : a[i] + lo_w;
            }
            for (int bz = lo[2]; bz <= hi[2]; bz++)
                for (int by = lo[1]; by <= hi[1]; by++)
                    for (int bx = lo[0]; bx <= hi[0]; bx++) {
                        int b[3] = {bx, by, bz};
                        if (bx == a[0] && by == a[1] && bz == a[2]) continue;
                        int bn = t.find(L, bx >> 3, by >> 3, bz >> 3);
                        if (bn < 0) continue;
                        bool leaf_b = nodes[bn].leaf_id >= 0;
                        int cls = classify(L, a, b, it2, leaf_a, leaf_b);  // symmetric in a, b
                        if (cls == 0 || cls == 4) continue;
                        long bi = (long)bn * 512 + local_of(bx & 7, by & 7, bz & 7);
                        const Mom<double>& P = w.mom[L][bi];
                        if (cls == 2) {
                            // C as the source of P's exact near pair
                            double r[3];
                            for (int i = 0; i < 3; i++) r[i] = P.X[i] - C.X[i];
                            double rr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                            long pl = (long)nodes[bn].leaf_id * 512 + local_of(bx & 7, by & 7, bz & 7);
                            double v = w1[pl] / rr;
                            for (int i = 0; i < 3; i++) v += w2[(pl / 512 * 3 + i) * 512 + pl % 512] * r[i] / (rr * rr * rr);
                            Mb[L][ci].m += -G * v;
                            continue;
                        }
                        // C as target of P, then C as source for P
                        m2l_reverse(C, P, G, am, Eb[L][ci], &Mb[L][ci], nullptr, !leaf_a);
                        m2l_reverse(P, C, G, am, Eb[L][bi], nullptr, &Mb[L][ci], !leaf_a);
                    }
        }
    }
    // M2M reverse, top-down
    for (int L = 0; L < t.Lmax; L++) {
        const auto& nodes = t.lev[L];
        long nc = (long)nodes.size() * 512;
#pragma omp parallel for schedule(static)
        for (long pi = 0; pi < nc; pi++) {
            const Node& nd = nodes[pi / 512];
            if (nd.leaf_id >= 0) continue;
            int l = (int)(pi % 512);
            int a[3] = {8 * nd.x + (l & 7), 8 * nd.y + ((l >> 3) & 7), 8 * nd.z + (l >> 6)};
            Mom<double> ch[8];
            long cix[8];
            MomBar cb[8];
            for (int c = 0; c < 8; c++) {
                cix[c] = t.cell(L + 1, 2 * a[0] + (c & 1), 2 * a[1] + ((c >> 1) & 1), 2 * a[2] + (c >> 2));
                ch[c] = w.mom[L + 1][cix[c]];
                zero_bar(cb[c]);
            }
            m2m_reverse(ch, 8, w.mom[L][pi], Mb[L][pi], cb);
            for (int c = 0; c < 8; c++) {
                MomBar& o = Mb[L + 1][cix[c]];
                o.m += cb[c].m;
                for (int i = 0; i < 3; i++) {
                    o.X[i] += cb[c].X[i];
                    for (int j = 0; j < 3; j++) {
                        o.M2[i][j] += cb[c].M2[i][j];
                        for (int k = 0; k < 3; k++) o.M3[i][j][k] += cb[c].M3[i][j][k];
                    }
                }
            }
        }
    }
    // leaf masses m = rho h^3 (leaf positions are constants)
    double Cc = self_term ? cube_self_constant() : 0.0;
    for (int L = 0; L <= t.Lmax; L++) {
        double h = t.h(L);
        for (long n = 0; n < (long)t.lev[L].size(); n++) {
            int leaf = t.lev[L][n].leaf_id;
            if (leaf < 0) continue;
            for (int l = 0; l < 512; l++) {
                long o = (long)leaf * 512 + l;
                drho[o] = Mb[L][n * 512 + l].m * h * h * h;
                if (self_term) drho[o] += -G * h * h * Cc * w1[o];
            }
        }
    }
    return ORC_OK;
}

void pack_mom(const Mom<double>& M, double* o) {
    o[0] = M.m;
    for (int i = 0; i < 3; i++) o[1 + i] = M.X[i];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            o[4 + 3 * i + j] = M.M2[i][j];
            for (int k = 0; k < 3; k++) o[13 + 9 * i + 3 * j + k] = M.M3[i][j][k];
        }
}
void unpack_mom(const double* o, Mom<double>& M) {
    M.m = o[0];
    for (int i = 0; i < 3; i++) M.X[i] = o[1 + i];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            M.M2[i][j] = o[4 + 3 * i + j];
            for (int k = 0; k < 3; k++) M.M3[i][j][k] = o[13 + 9 * i + 3 * j + k];
        }
}
void pack_loc(const Loc<double>& E, double* o) {
    o[0] = E.L0;
    for (int i = 0; i < 3; i++) o[1 + i] = E.L1[i];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            o[4 + 3 * i + j] = E.L2[i][j];
            for (int k = 0; k < 3; k++) o[13 + 9 * i + 3 * j + k] = E.L3[i][j][k];
        }
    for (int i = 0; i < 3; i++) o[40 + i] = E.ac[i];
}
void unpack_loc(const double* o, Loc<double>& E) {
    E.L0 = o[0];
    for (int i = 0; i < 3; i++) E.L1[i] = o[1 + i];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            E.L2[i][j] = o[4 + 3 * i + j];
            for (int k = 0; k < 3; k++) E.L3[i][j][k] = o[13 + 9 * i + 3 * j + k];
        }
    for (int i = 0; i < 3; i++) E.ac[i] = o[40 + i];
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (called through ctypes by the oracle's Python wrapper).
extern "C" {

int orc_set_threads(int n) {
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

// Full solve: phi [n_leaf][512], g [n_leaf][3][512] in the caller's leaf
// order, cell (i, j, k) of a leaf at i + 8 j + 64 k.  counts (optional):
// [0] far M2L pairs, [1] exact near pairs, [2] mixed near pairs (F3).
int orc_solve(int n_leaf, const int32_t* leaves, const double* origin, double size,
              const double* rho, double theta, double G, int am, int self_term, double* phi,
              double* g, int64_t* counts) {
    Tree t;
    int e = build_tree(n_leaf, leaves, origin, size, t);
    if (e) return e;
    return solve<double>(t, rho, theta, G, am, self_term, phi, g, nullptr, 0, counts);
}

// Solve for a sample of leaf cells only: sample[s] = leaf * 512 + cell;
// phi_s [n_sample], g_s [n_sample][3]; counts (optional) as in orc_solve,
// restricted to the pairs evaluated for the sampled cells and their ancestors.
int orc_solve_sample(int n_leaf, const int32_t* leaves, const double* origin, double size,
                     const double* rho, double theta, double G, int am, int self_term,
                     long n_sample, const int64_t* sample, double* phi_s, double* g_s,
                     int64_t* counts) {
    Tree t;
    int e = build_tree(n_leaf, leaves, origin, size, t);
    if (e) return e;
    return solve<double>(t, rho, theta, G, am, self_term, phi_s, g_s, sample, n_sample, counts);
}

// Forward-mode directional derivative of (phi, g) along v (same layout as rho).
int orc_solve_jvp(int n_leaf, const int32_t* leaves, const double* origin, double size,
                  const double* rho, const double* v, double theta, double G, int am,
                  int self_term, double* phi, double* g, double* dphi, double* dg) {
    Tree t;
    int e = build_tree(n_leaf, leaves, origin, size, t);
    if (e) return e;
    long n = (long)n_leaf * 512;
    std::vector<Dual> r(n), p(n), gg(3 * n);
    for (long i = 0; i < n; i++) r[i] = Dual(rho[i], v[i]);
    e = solve<Dual>(t, r.data(), theta, G, am, self_term, p.data(), gg.data(), nullptr, 0, nullptr);
    if (e) return e;
    for (long i = 0; i < n; i++) {
        phi[i] = p[i].v;
        dphi[i] = p[i].d;
    }
    for (long i = 0; i < 3 * n; i++) {
        g[i] = gg[i].v;
        dg[i] = gg[i].d;
    }
    return ORC_OK;
}

// O(N^2) direct summation over all leaf cells as point masses (O0).
int orc_direct(int n_leaf, const int32_t* leaves, const double* origin, double size,
               const double* rho, double G, double* phi, double* g) {
    Tree t;
    int e = build_tree(n_leaf, leaves, origin, size, t);
    if (e) return e;
    long n = (long)n_leaf * 512;
    std::vector<double> x(3 * n), m(n);
    for (int i = 0; i < n_leaf; i++) {
        int L = leaves[4 * i];
        double h = t.h(L);
        for (int l = 0; l < 512; l++) {
            int c[3] = {8 * leaves[4 * i + 1] + (l & 7), 8 * leaves[4 * i + 2] + ((l >> 3) & 7),
                        8 * leaves[4 * i + 3] + (l >> 6)};
            long q = (long)i * 512 + l;
            for (int a = 0; a < 3; a++) x[3 * q + a] = t.origin[a] + (c[a] + 0.5) * h;
            m[q] = rho[q] * h * h * h;
        }
    }
#pragma omp parallel for schedule(static)
    for (long a = 0; a < n; a++) {
        double p = 0.0, ga[3] = {0.0, 0.0, 0.0};
        for (long b = 0; b < n; b++) {
            if (b == a) continue;
            double r[3] = {x[3 * a] - x[3 * b], x[3 * a + 1] - x[3 * b + 1], x[3 * a + 2] - x[3 * b + 2]};
            double rr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            p += -G * m[b] / rr;
            for (int i = 0; i < 3; i++) ga[i] += -G * m[b] * r[i] / (rr * rr * rr);
        }
        phi[a] = p;
        long leaf = a / 512, l = a % 512;
        for (int i = 0; i < 3; i++) g[(leaf * 3 + i) * 512 + l] = ga[i];
    }
    return ORC_OK;
}

// Moments of every cell at level L (nodes in the oracle's own order, returned
// with their coordinates): out [n_nodes*512][40] = (m, X[3], M2[9], M3[27]),
// node_xyz [n_nodes][3].  Call with out = nullptr to get the node count.
long orc_level_moments(int n_leaf, const int32_t* leaves, const double* origin, double size,
                       const double* rho, int L, double* out, int32_t* node_xyz) {
    Tree t;
    int e = build_tree(n_leaf, leaves, origin, size, t);
    if (e) return e;
    if (L < 0 || L > t.Lmax) return ORC_BAD_LEAF;
    if (!out) return (long)t.lev[L].size();
    Work<double> w;
    upward(t, rho, w);
    for (long n = 0; n < (long)t.lev[L].size(); n++) {
        node_xyz[3 * n] = t.lev[L][n].x;
        node_xyz[3 * n + 1] = t.lev[L][n].y;
        node_xyz[3 * n + 2] = t.lev[L][n].z;
        for (int l = 0; l < 512; l++) pack_mom(w.mom[L][n * 512 + l], out + (n * 512 + l) * 40);
    }
    return (long)t.lev[L].size();
}

// Tree validation only (0 or a negative error code).
int orc_check_tree(int n_leaf, const int32_t* leaves) {
    Tree t;
    return build_tree(n_leaf, leaves, nullptr, 1.0, t);
}

// Primitives exposed for the tests.
// D tensors: out = D0 (1), D1 (3), D2 (9), D3 (27), D4 (81).
void orc_dtensor(const double* R, double* out) {
    DTens<double> D;
    double r[3] = {R[0], R[1], R[2]};
    dtensors(r, D);
    out[0] = D.D0;
    int o = 1;
    for (int i = 0; i < 3; i++) out[o++] = D.D1[i];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) out[o++] = D.D2[i][j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) out[o++] = D.D3[i][j][k];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) out[o++] = D.D4[i][j][k][l];
}

// Point masses -> single-cell moments through U1 + U2 (each point is a
// leaf-like moment set, combined by one M2M step).
void orc_p2m_m2m(int n, const double* pts, const double* m, double* out) {
    std::vector<Mom<double>> ch(n);
    for (int c = 0; c < n; c++) {
        zero_mom(ch[c]);
        ch[c].m = m[c];
        for (int i = 0; i < 3; i++) ch[c].X[i] = pts[3 * c + i];
    }
    Mom<double> P;
    m2m(ch.data(), n, P);
    pack_mom(P, out);
}

// U2 on packed moments: moms [n][40] -> out [40].
void orc_m2m(int n, const double* moms, double* out) {
    std::vector<Mom<double>> ch(n);
    for (int c = 0; c < n; c++) unpack_mom(moms + 40 * c, ch[c]);
    Mom<double> P;
    m2m(ch.data(), n, P);
    pack_mom(P, out);
}

// F1 + F2 on packed moments: out [43] = (L0, L1[3], L2[9], L3[27], ac[3]).
void orc_m2l(const double* momA, const double* momB, double G, int am, double* out) {
    Mom<double> A, B;
    unpack_mom(momA, A);
    unpack_mom(momB, B);
    Loc<double> E;
    zero_loc(E);
    m2l(A, B, G, am, E);
    pack_loc(E, out);
}

// D1 on packed expansions: out = shift of loc by delta (out is overwritten).
void orc_l2l(const double* loc, const double* delta, double* out) {
    Loc<double> P, C;
    unpack_loc(loc, P);
    zero_loc(C);
    double d[3] = {delta[0], delta[1], delta[2]};
    l2l(P, d, C);
    pack_loc(C, out);
}

double orc_cube_self_constant() { return cube_self_constant(); }

// Hand-written adjoint: drho = dJ/drho for J = sum (w1 phi + w2 . g);
// w1 [n_leaf][512], w2 [n_leaf][3][512], drho [n_leaf][512].
int orc_gradient(int n_leaf, const int32_t* leaves, const double* origin, double size,
                 const double* rho, double theta, double G, int am, int self_term,
                 const double* w1, const double* w2, double* drho) {
    Tree t;
    int e = build_tree(n_leaf, leaves, origin, size, t);
    if (e) return e;
    return gradient(t, rho, theta, G, am, self_term, w1, w2, drho);
}

// Reverse of one pair (test primitive): momA/momB packed as in orc_m2l,
// Ebar [43] = adjoint of the target expansion (L0, L1[3], L2[9], L3[27],
// ac[3]); outA/outB [40] = adjoints (m, X[3], M2[9], M3[27]).
void orc_m2l_reverse(const double* momA, const double* momB, double G, int am, const double* Ebar,
                     double* outA, double* outB) {
    Mom<double> A, B;
    unpack_mom(momA, A);
    unpack_mom(momB, B);
    Loc<double> E;
    unpack_loc(Ebar, E);
    MomBar bA, bB;
    zero_bar(bA);
    zero_bar(bB);
    m2l_reverse(A, B, G, am, E, &bA, &bB, true);
    double* outs[2] = {outA, outB};
    MomBar* bs[2] = {&bA, &bB};
    for (int q = 0; q < 2; q++) {
        double* o = outs[q];
        o[0] = bs[q]->m;
        for (int i = 0; i < 3; i++) o[1 + i] = bs[q]->X[i];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                o[4 + 3 * i + j] = bs[q]->M2[i][j];
                for (int k = 0; k < 3; k++) o[13 + 9 * i + 3 * j + k] = bs[q]->M3[i][j][k];
            }
    }
}

// D^(5) at R: out [243].
void orc_dtensor5(const double* R, double* out) {
    double D5[3][3][3][3][3];
    double r[3] = {R[0], R[1], R[2]};
    dtensor5(r, D5);
    std::memcpy(out, D5, sizeof(D5));
}

}  // extern "C"
