// Device-side building blocks shared by the stage, setup and reduction kernels.
//
// Notation (Duru, Fung & Williams, arXiv 2011.02600): state Q = (v, sigma) with
// sigma in Voigt order (xx, yy, zz, xy, xz, yz); metrics a[xi][eta] = J xi_eta
// (the basis e_xi = J grad xi of Section 2.2); coefficients 1/(rho J), lambda/J,
// mu/J so that dQ/dt = P~ (P~^-1 dQ/dt) needs no division (P~ = J^-1 P,
// Eq. S matrix).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sbp_coeffs.h"

namespace sbp {

// Field layout: [s][r][q], q contiguous, row pitch ldq, plane pitch ldq*nr,
// field stride fs.  In-field offsets fit in 32 bits (checked at grid creation).
struct Dims {
  int nq, nr, ns;
  int ldq;
  int plane;     // ldq * nr
  long long fs;  // field stride in elements
};

// A slab of a block decomposed along s: the local arrays hold the planes one device owns
// plus ghost planes copied from its neighbours (halo exchange).  ghost_lo/ghost_hi = 0 mean
// that the local end is a face of the whole block (closures and penalties apply there);
// k_offset is the block's index of local plane 0; ns_global = 0 means no decomposition.
struct SlabS {
  int ghost_lo = 0, ghost_hi = 0;
  int k_offset = 0;
  int ns_global = 0;
};

// Face kind of an interface between two blocks (the host's SBP_BC_INTERFACE).
constexpr int kBcInterface = 2;

// The other block's trace at an interface face (one per face; null when the face is no
// interface): 8 fields of the face's nodes, v (3), T = sigma n (3), Z_p, Z_s, each field a face
// array in the order of face_index; member b of a batch at other + b * 8 * n_face.
template <typename T>
struct IfaceArgs {
  const T* other[6];
  long long n_face[6];
};

// Index of a node on face xi (0: q faces, [k][j]; 1: r faces, [k][i]; 2: s faces, [j][i]).
__host__ __device__ __forceinline__ long long face_index(int xi, int i, int j, int k, int nq, int nr) {
  return xi == 0 ? (long long)k * nr + j : xi == 1 ? (long long)k * nq + i : (long long)j * nq + i;
}

enum StageMode : int {
  kModeRhs = 0,     // write dQ/dt to qout
  kModeStage = 1,   // dq <- A dq + dt L; qout <- q + B dq
  kModeStage0 = 2,  // same with A = 0 (dq is not read)
};

template <typename T>
struct StageArgs {
  const T* __restrict__ q;
  T* __restrict__ qout;
  T* __restrict__ dq;
  const T* __restrict__ met;
  const T* __restrict__ mat;
  Dims d;
  T rk_a, rk_b, dt;
  int mode;
  int bc_kind[6];
  T bc_gamma[6];
  T inv_h[3];       // N_xi - 1 (reference spacing 1/(N_xi - 1))
  T inv_h0[3];      // 1 / H_xi[0] = (N_xi - 1) / w_0
  T h[3];           // reference spacing 1 / (N_xi - 1)
  unsigned* status; // device status word (bit 8: a tile copy timed out)
  int nb;           // independent states processed together (shared metrics and coefficients)
  long long bstride;  // elements between consecutive states (9 fields)
  T* sclose;          // tiled kernel scratch: s-closure sums, 2 b 6 planes per state
  long long sc_bstride;  // elements between consecutive states' scratch
  // adjoint passes of the tiled kernel (q is then yhat = H^-1 P~ Wb_k, or U_k)
  const T* ubar_next;   // Ub_{k+1} (null: zero)
  T* ubar_out;          // Ub_k, or L^T w (mode kModeRhs)
  T* wbar;              // Wb_k, replaced by A_k Wb_k
  const T* yhat;        // H^-1 P~ Wb_k (the gradient pass reads it at faces)
  const double* rlmj;   // rho, lambda, mu, J (FP64)
  double* grad;         // gradient accumulators (FP64, 3 fields)
  SlabS slab;           // s-slab of a decomposed block (default: the whole block)
  IfaceArgs<T> ifc;     // the other blocks' traces at interface faces (none by default)
  T* yhat_next;         // L^T pass of stage k > 0 in an adjoint step: where the fused prep of stage
                        // k - 1 writes yhat_{k-1} (null: no fusion, Wb <- A_k Wb_k)
  T rk_b_next;          // B_{k-1} of that fused prep
  int map;              // 1: topography map (a_q = (a_q,x, 0, 0), a_r = (0, ar_ratio a_q,x, 0)); 0: general
  T ar_ratio;           // a_r,y / a_q,x of a topography map (L_x / L_y)
};

// Closure rows of D+ and D- (unit spacing), one private copy per translation unit; orders
// kTraditional + 2, 4, 6 are Table 2's central operators (both tables hold D).
#define SBP_DECLARE_TABLES(O, B, CW)                                   \
  static __constant__ double kDpD##O[B][CW] = SBP_DP##O##_ROWS;        \
  static __constant__ double kDmD##O[B][CW] = SBP_DM##O##_ROWS;        \
  static __constant__ float kDpF##O[B][CW] = SBP_DP##O##_ROWS;         \
  static __constant__ float kDmF##O[B][CW] = SBP_DM##O##_ROWS;
SBP_DECLARE_TABLES(2, 2, 4)
SBP_DECLARE_TABLES(3, 2, 4)
SBP_DECLARE_TABLES(4, 4, 7)
SBP_DECLARE_TABLES(5, 4, 7)
SBP_DECLARE_TABLES(6, 6, 10)
SBP_DECLARE_TABLES(7, 6, 10)
SBP_DECLARE_TABLES(102, 1, 3)
SBP_DECLARE_TABLES(104, 4, 6)
SBP_DECLARE_TABLES(106, 6, 9)
#undef SBP_DECLARE_TABLES

template <typename T, int O>
struct Tab;
#define SBP_TAB(T, SUF, O)                                                              \
  template <>                                                                           \
  struct Tab<T, O> {                                                                    \
    __device__ __forceinline__ static T p(int i, int c) { return kDp##SUF##O[i][c]; }   \
    __device__ __forceinline__ static T m(int i, int c) { return kDm##SUF##O[i][c]; }   \
  };
SBP_TAB(double, D, 2)
SBP_TAB(double, D, 3)
SBP_TAB(double, D, 4)
SBP_TAB(double, D, 5)
SBP_TAB(double, D, 6)
SBP_TAB(double, D, 7)
SBP_TAB(float, F, 2)
SBP_TAB(float, F, 3)
SBP_TAB(float, F, 4)
SBP_TAB(float, F, 5)
SBP_TAB(float, F, 6)
SBP_TAB(float, F, 7)
SBP_TAB(double, D, 102)
SBP_TAB(double, D, 104)
SBP_TAB(double, D, 106)
SBP_TAB(float, F, 102)
SBP_TAB(float, F, 104)
SBP_TAB(float, F, 106)
#undef SBP_TAB

// Row `pos` of D+ (PLUS) or D- on N nodes, unit spacing, applied through
// fn(node_index_along_axis, weight).  Interior rows are Table 1's stencil
// (alpha_j for D+, beta_j = -alpha_{-j} for D-); the b rows at each end are
// the closure tables, the right end by D+[N-1-i][N-1-j] = -D-[i][j].
template <typename T, int O, bool PLUS, class Fn>
__device__ __forceinline__ void apply_row(int pos, int N, Fn&& fn) {
  using C = OpCoef<O>;
  if (pos < C::b) {
#pragma unroll
    for (int c = 0; c < C::cw; ++c) {
      const T w = PLUS ? Tab<T, O>::p(pos, c) : Tab<T, O>::m(pos, c);
      if (w != T(0)) fn(c, w);
    }
  } else if (pos > N - 1 - C::b) {
    const int ii = N - 1 - pos;
#pragma unroll
    for (int c = 0; c < C::cw; ++c) {
      const T w = PLUS ? Tab<T, O>::m(ii, c) : Tab<T, O>::p(ii, c);
      if (w != T(0)) fn(N - 1 - c, -w);
    }
  } else {
    if (PLUS) {
#pragma unroll
      for (int j = -C::r; j <= C::q; ++j) fn(pos + j, T(C::alpha(j)));
    } else {
#pragma unroll
      for (int j = -C::q; j <= C::r; ++j) fn(pos + j, T(-C::alpha(-j)));
    }
  }
}

template <int O>
__host__ __device__ __forceinline__ double norm_weight(int pos, int N) {
  const int e = pos < N - 1 - pos ? pos : N - 1 - pos;
  return OpCoef<O>::w(e);
}

// Norm weight and its reciprocal in precision T, each a compile-time constant (no
// conversion or division at run time).
template <typename T, int O>
__device__ __forceinline__ T norm_weight_t(int pos, int N) {
  const int e = pos < N - 1 - pos ? pos : N - 1 - pos;
  constexpr T w0 = T(OpCoef<O>::w(0)), w1 = T(OpCoef<O>::w(1)), w2 = T(OpCoef<O>::w(2)), w3 = T(OpCoef<O>::w(3)),
              w4 = T(OpCoef<O>::w(4)), w5 = T(OpCoef<O>::w(5));
  return e == 0 ? w0 : e == 1 ? w1 : e == 2 ? w2 : e == 3 ? w3 : e == 4 ? w4 : e == 5 ? w5 : T(1);
}
template <typename T, int O>
__device__ __forceinline__ T norm_weight_inv_t(int pos, int N) {
  const int e = pos < N - 1 - pos ? pos : N - 1 - pos;
  constexpr T r0 = T(1.0 / OpCoef<O>::w(0)), r1 = T(1.0 / OpCoef<O>::w(1)), r2 = T(1.0 / OpCoef<O>::w(2)),
              r3 = T(1.0 / OpCoef<O>::w(3)), r4 = T(1.0 / OpCoef<O>::w(4)), r5 = T(1.0 / OpCoef<O>::w(5));
  return e == 0 ? r0 : e == 1 ? r1 : e == 2 ? r2 : e == 3 ? r3 : e == 4 ? r4 : e == 5 ? r5 : T(1);
}

// Flux rows of Eq. split_form with e_xi = a: F = sigma a.
template <typename T>
__device__ __forceinline__ void flux(const T a[3], const T s[6], T F[3]) {
  F[0] = a[0] * s[0] + a[1] * s[3] + a[2] * s[4];
  F[1] = a[0] * s[3] + a[1] * s[1] + a[2] * s[5];
  F[2] = a[0] * s[4] + a[1] * s[5] + a[2] * s[2];
}

// B_xi rows of Eq. split_form applied to dv = D+_xi v, accumulated into e.
template <typename T>
__device__ __forceinline__ void add_strain(const T a[3], const T dv[3], T e[6]) {
  e[0] += a[0] * dv[0];
  e[1] += a[1] * dv[1];
  e[2] += a[2] * dv[2];
  e[3] += a[1] * dv[0] + a[0] * dv[1];
  e[4] += a[2] * dv[0] + a[0] * dv[2];
  e[5] += a[2] * dv[1] + a[1] * dv[2];
}

// Penalty of one face at one face node, added to the velocity rows rv and the
// stress rows e of P~^-1 dQ/dt.
//  free (Eq. SAT_free_surface): rv += +-(1/H0) J|grad xi| T = +-(1/H0) sigma a
//    (+ at xi = 0, - at xi = 1);
//  general with gamma (Eq. SAT_General via Eq. penalty_terms and Eq. data_hat):
//    with Z equal on the two tangential directions the rotation R only splits
//    normal and tangential parts, G_n = ((1-g) Zp v_n -+ (1+g) T_n)/2 and
//    G_t = ((1-g) Zs v_t -+ (1+g) T_t)/2 (- at xi = 0, + at xi = 1),
//    G = G_n n + G_t, G~ = G_n/Zp n + G_t/Zs;
//    rv -= |a| G / H0,  e -= |a| (-+)(n (x) G~)_sym / H0.
template <typename T>
__device__ __forceinline__ void add_penalty(int side, int kind, T gamma, T inv_h0, const T v[3],
                                            const T s[6], const T a[3], T irhoJ, T lamJ, T muJ,
                                            T rv[3], T e[6]) {
  if (kind == 0) {
    T Fa[3];
    flux(a, s, Fa);
    const T sg = side == 0 ? inv_h0 : -inv_h0;
    rv[0] += sg * Fa[0];
    rv[1] += sg * Fa[1];
    rv[2] += sg * Fa[2];
    return;
  }
  const T an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  const T ian = T(1) / an;
  const T n[3] = {a[0] * ian, a[1] * ian, a[2] * ian};
  T Tr[3];
  flux(n, s, Tr);
  const T Zp = sqrt((lamJ + T(2) * muJ) / irhoJ);
  const T Zs = sqrt(muJ / irhoJ);
  const T iZp = T(1) / Zp, iZs = T(1) / Zs;
  const T vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  const T Tn = Tr[0] * n[0] + Tr[1] * n[1] + Tr[2] * n[2];
  const T sgT = side == 0 ? T(-1) : T(1);
  const T cv = T(0.5) * (T(1) - gamma);
  const T cT = T(0.5) * (T(1) + gamma) * sgT;
  const T Gn = cv * Zp * vn + cT * Tn;
  const T Gnp = Gn * iZp;
  T G[3], Gt[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T gt = cv * Zs * (v[c] - vn * n[c]) + cT * (Tr[c] - Tn * n[c]);
    G[c] = Gn * n[c] + gt;
    Gt[c] = Gnp * n[c] + gt * iZs;
  }
  const T f = an * inv_h0;
  rv[0] -= f * G[0];
  rv[1] -= f * G[1];
  rv[2] -= f * G[2];
  const T fs = side == 0 ? f : -f;   // e -= f * (side ? +1 : -1) * (n (x) G~)
  e[0] += fs * n[0] * Gt[0];
  e[1] += fs * n[1] * Gt[1];
  e[2] += fs * n[2] * Gt[2];
  e[3] += fs * (n[1] * Gt[0] + n[0] * Gt[1]);
  e[4] += fs * (n[2] * Gt[0] + n[0] * Gt[2]);
  e[5] += fs * (n[2] * Gt[1] + n[1] * Gt[2]);
}

// Interface penalty of one face node (Section 7.1's two blocks coupled weakly; the penalty of
// Eq. penalty_terms with the hat variables of a locked interface, velocity and traction
// continuous, both outgoing characteristics kept).  side 1: this block's face is at xi = 1
// (block "-"), side 0: at xi = 0 (block "+"); o: the other block's v, T, Z_p, Z_s at the node.
// With vhat from the two characteristics, G = Z (v - vhat) per part, G~ = G / Z = v - vhat:
//    vhat_n = (Z-_p v-_n - T-_n + Z+_p v+_n + T+_n) / (Z-_p + Z+_p), likewise tangential with Z_s,
//    rv -= |a| G / H0,  e -= |a| (-+)(n (x) G~)_sym / H0   (the signs of add_penalty).
template <typename T>
__device__ __forceinline__ void add_interface_penalty(int side, T inv_h0, const T v[3], const T s[6], const T a[3],
                                                      T irhoJ, T lamJ, T muJ, const T o[8], T rv[3], T e[6]) {
  const T an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  const T ian = T(1) / an;
  const T n[3] = {a[0] * ian, a[1] * ian, a[2] * ian};
  T Tr[3];
  flux(n, s, Tr);
  const T Zp = sqrt((lamJ + T(2) * muJ) / irhoJ);
  const T Zs = sqrt(muJ / irhoJ);
  // (this side, other side) as ("-", "+")
  const T* vm = side == 1 ? v : o;
  const T* Tm = side == 1 ? Tr : o + 3;
  const T* vp = side == 1 ? o : v;
  const T* Tp = side == 1 ? o + 3 : Tr;
  const T Zpm = side == 1 ? Zp : o[6], Zsm = side == 1 ? Zs : o[7];
  const T Zpp = side == 1 ? o[6] : Zp, Zsp = side == 1 ? o[7] : Zs;
  const T vmn = vm[0] * n[0] + vm[1] * n[1] + vm[2] * n[2], Tmn = Tm[0] * n[0] + Tm[1] * n[1] + Tm[2] * n[2];
  const T vpn = vp[0] * n[0] + vp[1] * n[1] + vp[2] * n[2], Tpn = Tp[0] * n[0] + Tp[1] * n[1] + Tp[2] * n[2];
  const T vhn = (Zpm * vmn - Tmn + Zpp * vpn + Tpn) / (Zpm + Zpp);
  const T vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  const T isz = T(1) / (Zsm + Zsp);
  T G[3], Gt[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T vht = (Zsm * (vm[c] - vmn * n[c]) - (Tm[c] - Tmn * n[c]) + Zsp * (vp[c] - vpn * n[c]) +
                   (Tp[c] - Tpn * n[c])) * isz;
    const T dt_ = (v[c] - vn * n[c]) - vht;   // tangential part of v - vhat
    const T dn = vn - vhn;                     // normal part
    Gt[c] = dn * n[c] + dt_;
    G[c] = Zp * dn * n[c] + Zs * dt_;
  }
  const T f = an * inv_h0;
  rv[0] -= f * G[0];
  rv[1] -= f * G[1];
  rv[2] -= f * G[2];
  const T fs = side == 0 ? f : -f;
  e[0] += fs * n[0] * Gt[0];
  e[1] += fs * n[1] * Gt[1];
  e[2] += fs * n[2] * Gt[2];
  e[3] += fs * (n[1] * Gt[0] + n[0] * Gt[1]);
  e[4] += fs * (n[2] * Gt[0] + n[0] * Gt[2]);
  e[5] += fs * (n[2] * Gt[1] + n[1] * Gt[2]);
}

// dQ/dt = P~ (rv, e): velocity rows / (rho J); stress rows C e / J.
template <typename T>
__device__ __forceinline__ void apply_P(const T rv[3], const T e[6], T irhoJ, T lamJ, T muJ, T d[9]) {
  d[0] = irhoJ * rv[0];
  d[1] = irhoJ * rv[1];
  d[2] = irhoJ * rv[2];
  const T tr = lamJ * (e[0] + e[1] + e[2]);
  const T m2 = T(2) * muJ;
  d[3] = tr + m2 * e[0];
  d[4] = tr + m2 * e[1];
  d[5] = tr + m2 * e[2];
  d[6] = muJ * e[3];
  d[7] = muJ * e[4];
  d[8] = muJ * e[5];
}

// Section 2.2: J and a[xi][eta] = J xi_eta at node t of the [s][r][q] enumeration from the node
// coordinates xyz (3 FP64 fields), into jmet (J, then the 9 metrics; FP64).  Coordinate
// derivatives use D_c = (D+ + D-)/2 along each axis.  Returns false where J <= 0.
template <int O>
// On a slab of a decomposed block (sl) node t enumerates the owned planes, and the s position and
// node count are the block's: the rows of D_c along s are the block's, their taps reaching into
// the ghost planes.
__device__ __forceinline__ bool metrics_at(const double* __restrict__ xyz, double* __restrict__ jmet, const Dims& d,
                                           long long t, SlabS sl = SlabS{}) {
  const int i = (int)(t % d.nq);
  const int j = (int)((t / d.nq) % d.nr);
  const int k = sl.ghost_lo + (int)(t / ((long long)d.nq * d.nr));
  const long long n0 = (long long)k * d.plane + (long long)j * d.ldq + i;
  const int pos[3] = {i, j, k + sl.k_offset};
  const int N[3] = {d.nq, d.nr, sl.ns_global > 0 ? sl.ns_global : d.ns};
  const long long stride[3] = {1, d.ldq, d.plane};
  double der[3][3];  // der[xi][c] = d x_c / d xi
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    double s[3] = {0, 0, 0};
    auto acc = [&](int c, double w) {
      const long long nb = n0 + (long long)(c - pos[xi]) * stride[xi];
      s[0] += 0.5 * w * xyz[nb];
      s[1] += 0.5 * w * xyz[d.fs + nb];
      s[2] += 0.5 * w * xyz[2 * d.fs + nb];
    };
    apply_row<double, O, true>(pos[xi], N[xi], acc);
    apply_row<double, O, false>(pos[xi], N[xi], acc);
    const double ih = (double)(N[xi] - 1);
    der[xi][0] = s[0] * ih;
    der[xi][1] = s[1] * ih;
    der[xi][2] = s[2] * ih;
  }
  // cross products: a_q = x_r x x_s, a_r = x_s x x_q, a_s = x_q x x_r (cofactors, Cramer's rule)
  double a[3][3];
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    const double* u = der[(xi + 1) % 3];
    const double* v = der[(xi + 2) % 3];
    a[xi][0] = u[1] * v[2] - u[2] * v[1];
    a[xi][1] = u[2] * v[0] - u[0] * v[2];
    a[xi][2] = u[0] * v[1] - u[1] * v[0];
  }
  const double J = der[0][0] * a[0][0] + der[0][1] * a[0][1] + der[0][2] * a[0][2];
  jmet[n0] = J;
#pragma unroll
  for (int xi = 0; xi < 3; ++xi)
#pragma unroll
    for (int c = 0; c < 3; ++c) jmet[(1 + 3 * xi + c) * d.fs + n0] = a[xi][c];
  return J > 0.0;
}

// Energy density of one node over a single division: with l = lambda/J, m = mu/J,
// r = 1/(rho J) and A = sum s_ii^2 + 2 sum s_ij^2,
//   rho J |v|^2 + J sigma^T S sigma = |v|^2 / r + (A (3 l + 2 m) - l tr^2) / ((3 l + 2 m) 2 m)
//                                  = (|v|^2 D + r (A (3 l + 2 m) - l tr^2)) / (r D),  D = (3 l + 2 m) 2 m.
// Evaluated in the state's precision (FP32 terms are summed in FP64).
template <typename T>
__device__ __forceinline__ T energy_density(const T v[3], const T s[6], T r, T l, T m) {
  const T v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const T tr = s[0] + s[1] + s[2];
  const T A = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + T(2) * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
  const T c = T(3) * l + T(2) * m;
  const T D = c * T(2) * m;
  return (v2 * D + r * (A * c - l * tr * tr)) / (r * D);
}

// Write the stage result for one node at in-field offset off.
template <typename T>
__device__ __forceinline__ void stage_epilogue(const StageArgs<T>& A, long long off, const T d[9],
                                               const T qc[9]) {
  const long long fs = A.d.fs;
  if (A.mode == kModeRhs) {
#pragma unroll
    for (int f = 0; f < 9; ++f) A.qout[f * fs + off] = d[f];
    return;
  }
#pragma unroll
  for (int f = 0; f < 9; ++f) {
    T dn = A.dt * d[f];
    if (A.mode == kModeStage) dn += A.rk_a * A.dq[f * fs + off];
    A.dq[f * fs + off] = dn;
    A.qout[f * fs + off] = qc[f] + A.rk_b * dn;
  }
}

// Contribution of axis xi to the raw operator at one node (in-field offset n0, position
// pos along the axis of N nodes, neighbour stride `stride`), read from global memory with
// every row of D+ and D- (interior stencil or closure):
//   rv += inv_h D-_xi (sigma a^xi),   e += B_xi(a^xi at the node) inv_h D+_xi v.
template <typename T, int O>
__device__ __forceinline__ void axis_operator_global(const T* __restrict__ q, const T* __restrict__ met,
                                                     long long fs, long long n0, int xi, int pos, int N,
                                                     long long stride, T inv_h, T rv[3], T e[6]) {
  const T* __restrict__ mx = met + (long long)(3 * xi) * fs;
  T f[3] = {T(0), T(0), T(0)};
  apply_row<T, O, false>(pos, N, [&](int c, T w) {
    const long long nb = n0 + (long long)(c - pos) * stride;
    const T a[3] = {mx[nb], mx[fs + nb], mx[2 * fs + nb]};
    T s[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) s[m] = q[(3 + m) * fs + nb];
    T F[3];
    flux(a, s, F);
    f[0] += w * F[0];
    f[1] += w * F[1];
    f[2] += w * F[2];
  });
  rv[0] += inv_h * f[0];
  rv[1] += inv_h * f[1];
  rv[2] += inv_h * f[2];
  T dv[3] = {T(0), T(0), T(0)};
  apply_row<T, O, true>(pos, N, [&](int c, T w) {
    const long long nb = n0 + (long long)(c - pos) * stride;
    dv[0] += w * q[nb];
    dv[1] += w * q[fs + nb];
    dv[2] += w * q[2 * fs + nb];
  });
  dv[0] *= inv_h;
  dv[1] *= inv_h;
  dv[2] *= inv_h;
  const T a0[3] = {mx[n0], mx[fs + n0], mx[2 * fs + n0]};
  add_strain(a0, dv, e);
}

// Penalty of face (xi, side) at one node: the boundary penalties of add_penalty, or the interface
// penalty with the other block's trace at the node (ifc; member b of a batch).
template <typename T>
__device__ __forceinline__ void face_penalty_at(int xi, int side, const int pos[3], const int N[3], const T a[3],
                                                const T qc[9], T irhoJ, T lamJ, T muJ, const int bc_kind[6],
                                                const T bc_gamma[6], const T inv_h0[3], T rv[3], T e[6],
                                                const IfaceArgs<T>* ifc, int member) {
  const int face = 2 * xi + side;
  if (bc_kind[face] == kBcInterface) {
    if (!ifc || !ifc->other[face]) return;  // refused on the host before any launch
    const long long nf = ifc->n_face[face];
    const T* src = ifc->other[face] + (long long)member * 8 * nf + face_index(xi, pos[0], pos[1], pos[2], N[0], N[1]);
    T o[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) o[c] = src[c * nf];
    add_interface_penalty<T>(side, inv_h0[xi], qc, qc + 3, a, irhoJ, lamJ, muJ, o, rv, e);
    return;
  }
  add_penalty<T>(side, bc_kind[face], bc_gamma[face], inv_h0[xi], qc, qc + 3, a, irhoJ, lamJ, muJ, rv, e);
}

// Penalties of every face the node lies on (positions pos, sizes N), in the order
// q = 0, q = 1, r = 0, r = 1, s = 0, s = 1.  a[xi] is a^xi at the node, qc its state.
template <typename T>
__device__ __forceinline__ void add_face_penalties(const int pos[3], const int N[3], const T a[3][3],
                                                   const T qc[9], T irhoJ, T lamJ, T muJ, const int bc_kind[6],
                                                   const T bc_gamma[6], const T inv_h0[3], T rv[3], T e[6],
                                                   const IfaceArgs<T>* ifc = nullptr, int member = 0) {
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    if (pos[xi] == 0)
      face_penalty_at<T>(xi, 0, pos, N, a[xi], qc, irhoJ, lamJ, muJ, bc_kind, bc_gamma, inv_h0, rv, e, ifc, member);
    if (pos[xi] == N[xi] - 1)
      face_penalty_at<T>(xi, 1, pos, N, a[xi], qc, irhoJ, lamJ, muJ, bc_kind, bc_gamma, inv_h0, rv, e, ifc, member);
  }
}

// Raw operator (P~^-1 dQ/dt: velocity rows rv, stress rows e, penalties included) of the
// state q at one node with in-field offset n0 and axis positions pos, using every row of
// D+ and D- (interior stencil or closure).  qc receives the node's own 9 values.
template <typename T, int O>
__device__ __forceinline__ void raw_operator_at(const T* __restrict__ q, const T* __restrict__ met,
                                                const T* __restrict__ mat, const Dims& d, long long n0,
                                                const int pos[3], const T inv_h[3], const T inv_h0[3],
                                                const int bc_kind[6], const T bc_gamma[6], T rv[3], T e[6],
                                                T qc[9], const IfaceArgs<T>* ifc = nullptr, int member = 0) {
  const long long fs = d.fs;
  const int N[3] = {d.nq, d.nr, d.ns};
  const long long stride[3] = {1, d.ldq, d.plane};
#pragma unroll
  for (int c = 0; c < 3; ++c) rv[c] = T(0);
#pragma unroll
  for (int c = 0; c < 6; ++c) e[c] = T(0);
#pragma unroll
  for (int xi = 0; xi < 3; ++xi)
    axis_operator_global<T, O>(q, met, fs, n0, xi, pos[xi], N[xi], stride[xi], inv_h[xi], rv, e);
#pragma unroll
  for (int f = 0; f < 9; ++f) qc[f] = q[f * fs + n0];
  const bool face = pos[0] == 0 || pos[0] == N[0] - 1 || pos[1] == 0 || pos[1] == N[1] - 1 || pos[2] == 0 ||
                    pos[2] == N[2] - 1;
  if (face) {
    T a[3][3];
#pragma unroll
    for (int xi = 0; xi < 3; ++xi)
#pragma unroll
      for (int c = 0; c < 3; ++c) a[xi][c] = met[(3 * xi + c) * fs + n0];
    add_face_penalties(pos, N, a, qc, mat[n0], mat[fs + n0], mat[2 * fs + n0], bc_kind, bc_gamma, inv_h0, rv, e,
                       ifc, member);
  }
}

struct Box {
  int i0, i1, j0, j1, k0, k1;
};
struct BoxList {
  int n;
  Box b[8];
  long long off[9];  // prefix sums of box sizes
};

}  // namespace sbp
