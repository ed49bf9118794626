// Tile geometry of the tiled stage kernel (kernels_tiled.cu): tile size and halo, the node
// range each tile owns along q and r, the launch order of the tiles, the per-thread rows of D-
// and D+ along q, and the closure-row sums along s.  Device code of the kernel; without nvcc the same source compiles as
// host C++, so that the index arithmetic can be checked for any grid size on a CPU.
#pragma once

#include "common.cuh"

namespace sbp {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int HX = 4;              // halo in the tile loads (>= q of every order)
constexpr int BXH = TX + 2 * HX;   // 40
constexpr int BYH = TY + 2 * HX;   // 16

// Tile `t` of `nt` along an axis of n nodes, tile width w: origin of its loads and the
// owned node range [own0, own1).  The last tile starts at n - w rounded up to `align`
// (never below 0); the one before it gives up the nodes from there on.
struct TileAxis {
  int origin, own0, own1;
};
__device__ __forceinline__ TileAxis tile_axis(int t, int nt, int n, int w, int align) {
  int last = n - w > 0 ? n - w : 0;
  last = (last + align - 1) / align * align;
  TileAxis a;
  a.origin = t == nt - 1 ? last : t * w;
  a.own0 = a.origin;
  a.own1 = t == nt - 1 ? n : (t == nt - 2 ? last : (t + 1) * w);
  return a;
}

// Launch order of the tiles of one s chunk: groups of kSwizzle tile columns (q), in each
// group q fastest, then r.  Blocks start in about launch order, so the tiles that share a
// halo row (r neighbours, kSwizzle launches apart) and a halo column (q neighbours, next to
// each other) run close together in time and the second reads the halo from L2; in plain
// row order r neighbours start a whole row of tiles apart, and on wide grids the halo has
// left L2 by then.
constexpr int kSwizzle = 12;
__device__ __forceinline__ void swizzle_tiles(int lin, int nbx, int nby, int& bx, int& by) {
  const int full = nbx / kSwizzle;                 // complete groups
  const int group = lin / (kSwizzle * nby);
  if (group < full) {
    const int rem = lin - group * kSwizzle * nby;
    by = rem / kSwizzle;
    bx = group * kSwizzle + rem % kSwizzle;
  } else {
    const int gw = nbx - full * kSwizzle;          // width of the last, narrower group
    const int rem = lin - full * kSwizzle * nby;
    by = rem / gw;
    bx = full * kSwizzle + rem % gw;
  }
}

constexpr int kMaxCW = 10;  // widest closure row (order 6)

// Halo on the low side over which the kernel forms the q and r fluxes: the interior stencil's
// reach q for the upwind operators; the whole loaded halo HX for the central operators
// (OpCoef<kTraditional + order>), where the last tile along an axis can own closure rows that
// reach node 0 from an origin beyond q.
template <int O>
__host__ __device__ constexpr int flux_halo() { return O > kTraditional ? HX : OpCoef<O>::q; }

// Per-thread q rows of a tile that owns closure nodes: the smem column of tap 0 for
// D- (of the flux tile) and D+ (of the state tile) and the weights of kMaxCW taps.
template <typename T>
struct QRows {
  T wm[kMaxCW][TX];
  T wp[kMaxCW][TX];
  int bm[TX];
  int bp[TX];
};

// Rows of D- and D+ along q for thread column tx of a tile with origin i0, as cw taps
// starting at a shared-memory column: the closure row (the cw nodes nearest the face)
// for a node within b of a q face, the interior stencil otherwise, zero weights for a
// column the tile does not own ([own0, own1)).  Every tap lies in the computed flux
// columns [HX - flux_halo, HX+TX+R) and state columns [0, BXH).
template <typename T, int O>
__device__ __forceinline__ void fill_q_rows(QRows<T>& Qr, int tx, int i0, int own0, int own1, int nq) {
  using C = OpCoef<O>;
  constexpr int BC = C::b, CW = C::cw, Q = C::q, R = C::r;
  const int i = i0 + tx;
  const bool owned = i >= own0 && i < own1;
  int bm, bp;
  T wm[CW], wp[CW];
  if (owned && i < BC) {
    bm = bp = HX - i0;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      wm[c] = Tab<T, O>::m(i, c);
      wp[c] = Tab<T, O>::p(i, c);
    }
  } else if (owned && i > nq - 1 - BC) {
    // tap t is node nq-cw+t, i.e. column cw-1-t of the mirrored closure row ii
    const int ii = nq - 1 - i;
    bm = bp = HX + nq - CW - i0;
#pragma unroll
    for (int t = 0; t < CW; ++t) {
      wm[t] = -Tab<T, O>::p(ii, CW - 1 - t);
      wp[t] = -Tab<T, O>::m(ii, CW - 1 - t);
    }
  } else {
    // interior stencil, placed so that all cw taps stay inside the computed columns
    const int dm = HX + tx - Q, dp = HX + tx - R;
    bm = min(dm, HX + TX + R - CW);
    bp = min(dp, BXH - CW);
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const int jm = bm + c - dm - Q;   // offset of this tap from the node for D-
      const int jp = bp + c - dp - R;   // and for D+
      wm[c] = owned && jm >= -Q && jm <= R ? T(-C::alpha(-jm)) : T(0);
      wp[c] = owned && jp >= -R && jp <= Q ? T(C::alpha(jp)) : T(0);
    }
  }
  Qr.bm[tx] = bm;
  Qr.bp[tx] = bp;
#pragma unroll
  for (int c = 0; c < kMaxCW; ++c) {
    Qr.wm[c][tx] = c < CW ? wm[c] : T(0);
    Qr.wp[c][tx] = c < CW ? wp[c] : T(0);
  }
}

// Closure-row sums of the b planes at one end of s (HI: the s = 1 end) for the node
// column col: for closure row r (plane r, or ns-1-r at the high end) and c = 0..2,
//   scratch[(e*b + r)*6 + c]     = sum_p D-[r][p] F_s,c(plane p)
//   scratch[(e*b + r)*6 + 3 + c] = sum_p D+[r][p] v_c(plane p)
// over the cw planes p nearest the face (unit spacing; rows of the high end by
// D+[N-1-i][N-1-j] = -D-[i][j]).  Each scratch row is a plane-sized array.
template <typename T, int O, bool HI>
__device__ __forceinline__ void s_closure_sums(const T* __restrict__ q, const T* __restrict__ met,
                                               const Dims& d, int col, T* __restrict__ scratch) {
  using C = OpCoef<O>;
  constexpr int BC = C::b;
  const long long fs = d.fs;
  T am[BC][3], ap[BC][3];
#pragma unroll
  for (int r = 0; r < BC; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) am[r][c] = ap[r][c] = T(0);
#pragma unroll
  for (int p = 0; p < C::cw; ++p) {
    const long long off = (long long)(HI ? d.ns - 1 - p : p) * d.plane + col;
    T v[3], sg[6], a[3], F[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = __ldg(q + c * fs + off);
#pragma unroll
    for (int c = 0; c < 6; ++c) sg[c] = __ldg(q + (3 + c) * fs + off);
#pragma unroll
    for (int c = 0; c < 3; ++c) a[c] = __ldg(met + (6 + c) * fs + off);
    flux(a, sg, F);
#pragma unroll
    for (int r = 0; r < BC; ++r) {
      const T wm = HI ? -Tab<T, O>::p(r, p) : Tab<T, O>::m(r, p);
      const T wp = HI ? -Tab<T, O>::m(r, p) : Tab<T, O>::p(r, p);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        am[r][c] += wm * F[c];
        ap[r][c] += wp * v[c];
      }
    }
  }
  T* out = scratch + (long long)(HI ? BC : 0) * 6 * d.plane + col;
#pragma unroll
  for (int r = 0; r < BC; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      out[(long long)(r * 6 + c) * d.plane] = am[r][c];
      out[(long long)(r * 6 + 3 + c) * d.plane] = ap[r][c];
    }
}

}  // namespace sbp
