// Tiled stage kernel over the whole grid.
//
// Work layout: a block owns a TX x TY tile of the (q, r) plane and marches along
// s through a chunk of planes.  Tiles start at multiples of TX and TY except the
// last along each axis, which is moved back so that it ends at the grid's edge
// (its start rounded up to a multiple of 4 along q, so that every tile load starts
// on a 16-byte boundary); the nodes it shares with the tile before it belong to it.
// Every closure row of D+ and D- along q and r then finds all of its taps in the
// tile that owns the node.
//   * Plane data arrive by TMA, one plane ahead, into a two-stage shared-memory
//     ring: the 9 state fields with a halo of HX nodes on q and r, a_q with a q
//     halo, a_r with an r halo, a_s and the coefficients on the tile.  One
//     elected thread issues the copies; an mbarrier per stage counts the bytes.
//   * Each plane, the fluxes F_q = sigma a_q and F_r = sigma a_r are formed on the
//     tile and its halo into a double-buffered flux tile; one block barrier per
//     plane publishes them and frees the stage the next copy will overwrite.
//   * q and r derivatives read the flux and velocity tiles (interior stencil, or
//     the closure row of a node within b of the face).  s derivatives use
//     per-thread register queues of F_s = sigma a_s (planes k-q..k+r) and v
//     (planes k-r..k+q), fed by direct loads of the lead planes.
//   * The b closure planes at each end of s all combine the same cw planes: a block
//     whose chunk reaches them first streams those planes once per thread and
//     forms the closure-row sums of every closure plane together, into a scratch
//     buffer that the same thread reads back when it gets to the plane.
//   * Nodes on a face add the face's penalty (free surface or characteristic SAT).
// The stage update (2N-storage Runge-Kutta) is fused in the epilogue.  Tiles of one s
// chunk launch in groups of tile columns (swizzle_tiles) so that tiles sharing halos run
// together and read them from L2.  The same kernel, templated on a pass kind, also runs
// the two stencil passes of the discrete adjoint (L^T on yhat, the material gradient on
// U_k) with their own epilogues; the L^T pass of an adjoint step can also form the next
// stage's pointwise prep (Wb and yhat) in its epilogue.  A second template argument selects
// the metric storage: MAP 0 reads the nine metric components; MAP 1, for topography maps
// (a_q and a_r along x and y only), reads a_q,x with both halos and a_s; MAP 2, the forward
// stage on such maps, also takes the RK register's tile in the same copy as the plane.
#include "adjoint_terms.cuh"
#include "common.cuh"
#include "launch.h"
#include "tile_map.cuh"
#include "tma.cuh"

namespace sbp {

constexpr unsigned kWaitLimit = 1u << 24;  // polls (with 64 ns sleeps) before giving up: about a second

// Metric storage the kernel reads.  MAP 0: the general curvilinear map, all nine a_xi.
// MAP 1: a topography map x = L_x q, y = L_y r, z = z(q, r, s), where a_q = (J / L_x, 0, 0) and
// a_r = (0, J / L_y, 0) = (0, c a_q,x, 0) with the constant c = L_x / L_y: only a_q,x (field 0,
// with halos on q and r) and a_s are read, 4 metric fields instead of 9.
template <typename T, int MAP>
struct Stage;
template <typename T>
struct Stage<T, 0> {
  T state[9][BYH][BXH];
  T aq[3][TY][BXH];
  T ar[3][BYH][TX];
  T as[3][TY][TX];
  T mat[3][TY][TX];
};
template <typename T>
struct Stage<T, 1> {
  T state[9][BYH][BXH];
  T jq[BYH][BXH];  // a_q,x on the tile and both halos
  T as[3][TY][TX];
  T mat[3][TY][TX];
};
// MAP 2: the topography map's forward stage, which also takes the RK register's tile with the
// plane (stages 1-4 of a step); the adjoint passes keep MAP 1 and the smaller stage.
template <typename T>
struct Stage<T, 2> : Stage<T, 1> {
  T dq[9][TY][TX];
};

// a_q at flux-tile row `row` (0..TY-1), smem column `col` (0..BXH-1); a_r at r-halo row `row`
// (0..BYH-1), column `col` (0..TX-1).
template <typename T>
__device__ __forceinline__ void aq_at(const Stage<T, 0>& st, int row, int col, T c_r, T a[3]) {
  (void)c_r;
  a[0] = st.aq[0][row][col];
  a[1] = st.aq[1][row][col];
  a[2] = st.aq[2][row][col];
}
template <typename T>
__device__ __forceinline__ void aq_at(const Stage<T, 1>& st, int row, int col, T c_r, T a[3]) {
  (void)c_r;
  a[0] = st.jq[HX + row][col];
  a[1] = T(0);
  a[2] = T(0);
}
template <typename T>
__device__ __forceinline__ void ar_at(const Stage<T, 0>& st, int row, int col, T c_r, T a[3]) {
  (void)c_r;
  a[0] = st.ar[0][row][col];
  a[1] = st.ar[1][row][col];
  a[2] = st.ar[2][row][col];
}
template <typename T>
__device__ __forceinline__ void ar_at(const Stage<T, 1>& st, int row, int col, T c_r, T a[3]) {
  a[0] = T(0);
  a[1] = c_r * st.jq[row][HX + col];
  a[2] = T(0);
}

// The RK register at the thread's node from the tile copy (MAP 2 only).
template <typename T>
__device__ __forceinline__ T dq_at(const Stage<T, 0>&, int, int, int) {
  return T(0);
}
template <typename T>
__device__ __forceinline__ T dq_at(const Stage<T, 1>&, int, int, int) {
  return T(0);
}
template <typename T>
__device__ __forceinline__ T dq_at(const Stage<T, 2>& st, int f, int ty, int tx) {
  return st.dq[f][ty][tx];
}

// Fluxes F_q = sigma a_q, F_r = sigma a_r and the strain rows of one axis; MAP 1, 2 skip the
// products with the components that vanish.
template <int MAP, typename T>
__device__ __forceinline__ void flux_q(const T a[3], const T s[6], T F[3]) {
  if constexpr (MAP >= 1) {
    F[0] = a[0] * s[0];
    F[1] = a[0] * s[3];
    F[2] = a[0] * s[4];
  } else {
    flux(a, s, F);
  }
}
template <int MAP, typename T>
__device__ __forceinline__ void flux_r(const T a[3], const T s[6], T F[3]) {
  if constexpr (MAP >= 1) {
    F[0] = a[1] * s[3];
    F[1] = a[1] * s[1];
    F[2] = a[1] * s[5];
  } else {
    flux(a, s, F);
  }
}
template <int MAP, typename T>
__device__ __forceinline__ void strain_q(const T a[3], const T dv[3], T e[6]) {
  if constexpr (MAP >= 1) {
    e[0] += a[0] * dv[0];
    e[3] += a[0] * dv[1];
    e[4] += a[0] * dv[2];
  } else {
    add_strain(a, dv, e);
  }
}
template <int MAP, typename T>
__device__ __forceinline__ void strain_r(const T a[3], const T dv[3], T e[6]) {
  if constexpr (MAP >= 1) {
    e[1] += a[1] * dv[1];
    e[3] += a[1] * dv[0];
    e[5] += a[1] * dv[2];
  } else {
    add_strain(a, dv, e);
  }
}

template <typename T>
struct FluxTiles {
  T fq[3][TY][BXH];
  T fr[3][BYH][TX];
};

template <typename T, int MAP>
struct TiledShared {
  Stage<T, MAP> st[2];
  FluxTiles<T> f[2];
  QRows<T> qrows;
  unsigned long long bar[2];
};

template <typename T>
constexpr int tiled_min_blocks() { return sizeof(T) == 4 ? 2 : 1; }

// with_dq (MAP 2): the RK register's box comes with the plane (the member Stage<T, 2> adds).
template <typename T, int MAP>
__device__ __forceinline__ void issue_plane(TiledShared<T, MAP>& S, int stage, const TmaSet& tm, int i0, int j0,
                                            int k, int member, bool with_dq) {
  unsigned long long* bar = &S.bar[stage];
  Stage<T, MAP>& st = S.st[stage];
  if constexpr (MAP == 2) {
    constexpr unsigned dq_bytes = (unsigned)sizeof(st.dq);
    mbar_expect_tx(bar, (unsigned)sizeof(Stage<T, MAP>) - (with_dq ? 0u : dq_bytes));
    if (with_dq) tma_load_4d(&st.dq[0][0][0], &tm.dq, i0, j0, k, 9 * member, bar);
  } else {
    (void)with_dq;
    mbar_expect_tx(bar, (unsigned)sizeof(Stage<T, MAP>));
  }
  tma_load_4d(&st.state[0][0][0], &tm.state, i0 - HX, j0 - HX, k, 9 * member, bar);
  if constexpr (MAP >= 1) {
    tma_load_4d(&st.jq[0][0], &tm.met_j, i0 - HX, j0 - HX, k, 0, bar);
  } else {
    tma_load_4d(&st.aq[0][0][0], &tm.met_q, i0 - HX, j0, k, 0, bar);
    tma_load_4d(&st.ar[0][0][0], &tm.met_r, i0, j0 - HX, k, 3, bar);
  }
  tma_load_4d(&st.as[0][0][0], &tm.met_s, i0, j0, k, 6, bar);
  tma_load_4d(&st.mat[0][0][0], &tm.mat, i0, j0, k, 0, bar);
}

// KIND 0: the forward stage.  KIND 1: the adjoint's L^T pass on q = yhat (-H times the
// forward rows, face terms of the transposes; Ub and Wb updated).  KIND 2: the material
// gradient pass on q = U_k (forward rows and penalties contracted with Wb_k).
template <typename T, int O, int KIND, int MAP>
__global__ void __launch_bounds__(TX* TY, tiled_min_blocks<T>())
    stage_tiled_kernel(StageArgs<T> A, int chunk, const __grid_constant__ TmaSet tm) {
  using C = OpCoef<O>;
  constexpr int R = C::r;    // D+ reaches -R..+Q, D- reaches -Q..+R
  constexpr int Q = C::q;
  constexpr int NV = R + Q + 1;
  constexpr int BC = C::b;   // closure rows at each end of an axis
  constexpr int CW = C::cw;  // columns of a closure row
  static_assert(CW <= TY + R && CW <= TX + R && BC <= TY, "closure rows must fit the first tile");
  static_assert(Q <= HX && R <= HX, "halo too small");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TiledShared<T, MAP>& S = *reinterpret_cast<TiledShared<T, MAP>*>(smem_raw);
  const T c_r = A.ar_ratio;  // MAP 1, 2: a_r,y / a_q,x

  const Dims d = A.d;
  const long long fs = d.fs;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  int bx, by;
  swizzle_tiles(blockIdx.x + gridDim.x * blockIdx.y, gridDim.x, gridDim.y, bx, by);
  const TileAxis ax = tile_axis(bx, gridDim.x, d.nq, TX, 4);
  const TileAxis ay = tile_axis(by, gridDim.y, d.nr, TY, 1);
  const int i0 = ax.origin, j0 = ay.origin;
  const int i = i0 + tx, j = j0 + ty;
  // blockIdx.z = chunk + nchunks * member (a batch of independent states).  The computed
  // planes are [klo, khi): the whole local array but a slab's ghost planes.
  const int klo = A.slab.ghost_lo, khi = d.ns - A.slab.ghost_hi;
  const bool face_lo = A.slab.ghost_lo == 0, face_hi = A.slab.ghost_hi == 0;
  const int nchunks = gridDim.z / A.nb;
  const int member = blockIdx.z / nchunks;
  const int kb = klo + (blockIdx.z % nchunks) * chunk;
  const int ke = min(khi, kb + chunk);
  const bool active = i >= ax.own0 && i < ax.own1 && j >= ay.own0 && j < ay.own1;
  // a tile owning nodes within b of a q face takes its q rows from a per-thread table
  const bool q_edge = ax.own0 < BC || ax.own1 > d.nq - BC;
  const bool r_close = j < BC || j > d.nr - 1 - BC;
  const bool qr_face = i == 0 || i == d.nq - 1 || j == 0 || j == d.nr - 1;
  const T ihq = A.inv_h[0], ihr = A.inv_h[1], ihs = A.inv_h[2];
  const long long boff = (long long)member * A.bstride;
  const T* __restrict__ q = A.q + boff;
  T* __restrict__ qout = A.qout + boff;
  T* __restrict__ dqm = A.dq + (A.mode == kModeRhs ? 0 : boff);
  T* __restrict__ scl = A.sclose + (long long)member * A.sc_bstride;
  const T* __restrict__ met = A.met;
  // this member's adjoint buffers (the adjoint passes; the gradient is shared by the members)
  const T* ub_next = A.ubar_next ? A.ubar_next + boff : nullptr;
  T* ub_out = A.ubar_out ? A.ubar_out + boff : nullptr;
  T* wbm = A.wbar ? A.wbar + boff : nullptr;
  const T* yhm = A.yhat ? A.yhat + boff : nullptr;
  const int col = j * d.ldq + i;
  // node offsets within a field as 32-bit indices from per-field base pointers (a field holds
  // fewer than 2^31 elements: the host refuses larger grids)
  auto fld = [&](const T* p, int c) -> const T* { return p + c * fs; };
  auto fldw = [&](T* p, int c) -> T* { return p + c * fs; };

  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
  }
  if (q_edge && ty == 0) fill_q_rows<T, O>(S.qrows, tx, i0, ax.own0, ax.own1, d.nq);  // read after the first plane's barrier
  __syncthreads();
  // the topography-map variant's stages read the RK register from the tile copy
  constexpr bool kDqTile = MAP == 2;
  const bool dq_tma = kDqTile && A.mode == kModeStage;
  if (tid == 0) issue_plane(S, 0, tm, i0, j0, kb, member, dq_tma);
  // closure-row sums of the s closure planes this chunk reaches (while the first copy flies)
  if (active && face_lo && kb < BC) s_closure_sums<T, O, false>(q, met, d, col, scl);
  if (active && face_hi && ke > d.ns - BC) s_closure_sums<T, O, true>(q, met, d, col, scl);

  auto ld = [&](const T* p, unsigned off) -> T { return active ? __ldg(p + off) : T(0); };
  // streamed once per launch (the RK register): evict-first in the caches
  auto ld_stream = [&](const T* p, unsigned off) -> T { return active ? __ldcs(p + off) : T(0); };
  // plane kk of field c of p at this thread's column; zero outside the grid
  auto ldk = [&](const T* p, int c, int kk) -> T {
    return active && kk >= 0 && kk < d.ns ? __ldg(fld(p, c) + ((unsigned)kk * (unsigned)d.plane + (unsigned)col))
                                          : T(0);
  };
  T vq[NV][3];  // v at planes k-R .. k+Q
  T fq[NV][3];  // F_s at planes k-Q .. k+R
#pragma unroll
  for (int m = 0; m < NV - 1; ++m) {
#pragma unroll
    for (int c = 0; c < 3; ++c) vq[m][c] = ldk(q, c, kb - R + m);
  }
#pragma unroll
  for (int m = 0; m < NV - 1; ++m) {
    T s[6], a[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c] = ldk(q, 3 + c, kb - Q + m);
#pragma unroll
    for (int c = 0; c < 3; ++c) a[c] = ldk(met, 6 + c, kb - Q + m);
    flux(a, s, fq[m]);
  }

  // lead values (v at k+Q, sigma and a_s at k+R) staged one plane ahead
  T lv[3], ls[6], la[3];
  auto load_lead = [&](int k) {
#pragma unroll
    for (int c = 0; c < 3; ++c) lv[c] = ldk(q, c, k + Q);
#pragma unroll
    for (int c = 0; c < 6; ++c) ls[c] = ldk(q, 3 + c, k + R);
#pragma unroll
    for (int c = 0; c < 3; ++c) la[c] = ldk(met, 6 + c, k + R);
  };
  load_lead(kb);

  for (int it = 0, k = kb; k < ke; ++it, ++k) {
    const int sidx = it & 1;
    const unsigned phase = (it >> 1) & 1;
    const unsigned off = (unsigned)k * (unsigned)d.plane + (unsigned)col;
    // the epilogue's own inputs at this node, fetched before the tile wait so that their
    // latency overlaps the plane's derivatives: the RK register (forward stage), Ub_{k+1} and
    // Wb_k (L^T pass), Wb_k, rho and J (gradient pass)
    T dqi[9], pre[9];
    double rj[2];
    if (KIND == 0 && !kDqTile && A.mode == kModeStage) {
#pragma unroll
      for (int c = 0; c < 9; ++c) dqi[c] = ld_stream(fld(dqm, c), off);
    }
    if (KIND == 1 && A.mode != kModeRhs) {
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        dqi[c] = ub_next ? ld(fld(ub_next, c), off) : T(0);
        pre[c] = ld(fld(wbm, c), off);
      }
    }
    if (KIND == 2) {
#pragma unroll
      for (int c = 0; c < 9; ++c) pre[c] = ld(fld(wbm, c), off);
      rj[0] = active ? __ldg(A.rlmj + off) : 0.0;
      rj[1] = active ? __ldg(A.rlmj + 3 * fs + off) : 0.0;
    }

    // Each thread waits for the plane's copy with a bounded wait; the block decides together
    // at the plane's barrier below (__syncthreads_or), so that either every thread goes on or
    // every thread leaves.  Until then a thread whose wait gave up only reads shared memory at
    // fixed in-bounds indices.
    const bool landed = mbar_wait_bounded(&S.bar[sidx], phase, kWaitLimit);
    const Stage<T, MAP>& st = S.st[sidx];
    FluxTiles<T>& F = S.f[sidx];
    // fluxes on the tile and its halo: F_q at columns -QF..TX-1+R, F_r at rows -QF..TY-1+R
    constexpr int QF = flux_halo<O>();
    for (int t = tid; t < TY * (QF + R + TX); t += TX * TY) {
      const int row = t / (QF + R + TX);
      const int cc = HX - QF + t % (QF + R + TX);
      T a[3], s[6];
      aq_at(st, row, cc, c_r, a);
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c] = st.state[3 + c][HX + row][cc];
      T Fv[3];
      flux_q<MAP>(a, s, Fv);
#pragma unroll
      for (int c = 0; c < 3; ++c) F.fq[c][row][cc] = Fv[c];
    }
    for (int t = tid; t < TX * (QF + R + TY); t += TX * TY) {
      const int cl = t % TX;
      const int rr = HX - QF + t / TX;
      T a[3], s[6];
      ar_at(st, rr, cl, c_r, a);
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c] = st.state[3 + c][rr][HX + cl];
      T Fv[3];
      flux_r<MAP>(a, s, Fv);
#pragma unroll
      for (int c = 0; c < 3; ++c) F.fr[c][rr][cl] = Fv[c];
    }
    if (__syncthreads_or(!landed)) {
      // The plane's copy did not complete in time for some thread (it is the only copy in
      // flight: the next plane's is issued below).  Record it and leave together; the host sees
      // SBP_STATUS_TIMEOUT.  The outstanding copy is abandoned.
      if (tid == 0) atomicOr(A.status, 8u);
      return;
    }
    if (tid == 0 && k + 1 < ke) {
      fence_proxy_async_smem();
      issue_plane(S, sidx ^ 1, tm, i0, j0, k + 1, member, dq_tma);
    }

    T rv[3] = {T(0), T(0), T(0)};
    T e[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T dv[3];
    // q
    if (!q_edge) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T sf = T(0), sv = T(0);
#pragma unroll
        for (int jj = -Q; jj <= R; ++jj) sf += T(-C::alpha(-jj)) * F.fq[c][ty][HX + tx + jj];
#pragma unroll
        for (int jj = -R; jj <= Q; ++jj) sv += T(C::alpha(jj)) * st.state[c][HX + ty][HX + tx + jj];
        rv[c] += ihq * sf;
        dv[c] = ihq * sv;
      }
    } else {
      const int bm = S.qrows.bm[tx], bp = S.qrows.bp[tx];
      T sf[3] = {T(0), T(0), T(0)}, sv[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const T wm = S.qrows.wm[c][tx], wp = S.qrows.wp[c][tx];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          sf[m] += wm * F.fq[m][ty][bm + c];
          sv[m] += wp * st.state[m][HX + ty][bp + c];
        }
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        rv[m] += ihq * sf[m];
        dv[m] = ihq * sv[m];
      }
    }
    {
      T a[3];
      aq_at(st, ty, HX + tx, c_r, a);
      strain_q<MAP>(a, dv, e);
    }
    // r
    if (!r_close) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T sf = T(0), sv = T(0);
#pragma unroll
        for (int jj = -Q; jj <= R; ++jj) sf += T(-C::alpha(-jj)) * F.fr[c][HX + ty + jj][tx];
#pragma unroll
        for (int jj = -R; jj <= Q; ++jj) sv += T(C::alpha(jj)) * st.state[c][HX + ty + jj][HX + tx];
        rv[c] += ihr * sf;
        dv[c] = ihr * sv;
      }
      T a[3];
      ar_at(st, HX + ty, tx, c_r, a);
      strain_r<MAP>(a, dv, e);
    } else if (active) {
      // closure row of a node within b of an r face (whole warps: the row is uniform)
      const bool lo = j < BC;
      const int row = lo ? j : d.nr - 1 - j;
      T sf[3] = {T(0), T(0), T(0)}, sv[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const int rr = HX + (lo ? c : d.nr - 1 - c) - j0;
        const T wm = lo ? Tab<T, O>::m(row, c) : -Tab<T, O>::p(row, c);
        const T wp = lo ? Tab<T, O>::p(row, c) : -Tab<T, O>::m(row, c);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          sf[m] += wm * F.fr[m][rr][tx];
          sv[m] += wp * st.state[m][rr][HX + tx];
        }
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        rv[m] += ihr * sf[m];
        dv[m] = ihr * sv[m];
      }
      T a[3];
      ar_at(st, HX + ty, tx, c_r, a);
      strain_r<MAP>(a, dv, e);
    }
    // push this plane's lead values (loaded one plane earlier), then fetch the next plane's, so
    // that their latency overlaps the s derivatives, the epilogue and the next plane's q and r
    // derivatives
#pragma unroll
    for (int c = 0; c < 3; ++c) vq[NV - 1][c] = lv[c];
    flux(la, ls, fq[NV - 1]);
    if (k + 1 < ke) load_lead(k + 1);
    // s (closure rows only within b of a face of the whole block)
    if ((k >= BC || !face_lo) && (k <= d.ns - 1 - BC || !face_hi)) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T sf = T(0), sv = T(0);
#pragma unroll
        for (int jj = -Q; jj <= R; ++jj) sf += T(-C::alpha(-jj)) * fq[Q + jj][c];
#pragma unroll
        for (int jj = -R; jj <= Q; ++jj) sv += T(C::alpha(jj)) * vq[R + jj][c];
        rv[c] += ihs * sf;
        dv[c] = ihs * sv;
      }
      const T a[3] = {st.as[0][ty][tx], st.as[1][ty][tx], st.as[2][ty][tx]};
      add_strain(a, dv, e);
    } else if (active) {
      // closure plane: the sums formed before the march
      const T* src = scl + (long long)((k < BC ? k : BC + d.ns - 1 - k) * 6) * d.plane + col;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        rv[m] += ihs * src[m * d.plane];
        dv[m] = ihs * src[(3 + m) * d.plane];
      }
      const T a[3] = {st.as[0][ty][tx], st.as[1][ty][tx], st.as[2][ty][tx]};
      add_strain(a, dv, e);
    }

    if (active && KIND == 0) {
      T qc[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) qc[c] = st.state[c][HX + ty][HX + tx];
      if (qr_face || k == 0 || k == d.ns - 1) {
        const int pos[3] = {i, j, k};
        const int N[3] = {d.nq, d.nr, d.ns};
        T a[3][3];
        aq_at(st, ty, HX + tx, c_r, a[0]);
        ar_at(st, HX + ty, tx, c_r, a[1]);
#pragma unroll
        for (int c = 0; c < 3; ++c) a[2][c] = st.as[c][ty][tx];
        add_face_penalties(pos, N, a, qc, st.mat[0][ty][tx], st.mat[1][ty][tx], st.mat[2][ty][tx], A.bc_kind,
                           A.bc_gamma, A.inv_h0, rv, e, &A.ifc, member);
      }
      T dd[9];
      apply_P(rv, e, st.mat[0][ty][tx], st.mat[1][ty][tx], st.mat[2][ty][tx], dd);
      if (A.mode == kModeRhs) {
#pragma unroll
        for (int f = 0; f < 9; ++f) fldw(qout, f)[off] = dd[f];
      } else {
#pragma unroll
        for (int f = 0; f < 9; ++f) {
          T dn = A.dt * dd[f];
          if (A.mode == kModeStage) {
            if constexpr (kDqTile)
              dn += A.rk_a * dq_at(st, f, ty, tx);
            else
              dn += A.rk_a * dqi[f];
          }
          __stcs(fldw(dqm, f) + off, dn);                    // read again one stage later
          __stcs(fldw(qout, f) + off, qc[f] + A.rk_b * dn);
        }
      }
    } else if (active) {
      T qc[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) qc[c] = st.state[c][HX + ty][HX + tx];
      const bool face = qr_face || k == 0 || k == d.ns - 1;
      const int pos[3] = {i, j, k};
      const int N[3] = {d.nq, d.nr, d.ns};
      const T irhoJ = st.mat[0][ty][tx], lamJ = st.mat[1][ty][tx], muJ = st.mat[2][ty][tx];
      T a[3][3];
      if (face) {
        aq_at(st, ty, HX + tx, c_r, a[0]);
        ar_at(st, HX + ty, tx, c_r, a[1]);
#pragma unroll
        for (int c = 0; c < 3; ++c) a[2][c] = st.as[c][ty][tx];
      }
      if (KIND == 2 && face)
        add_face_penalties(pos, N, a, qc, irhoJ, lamJ, muJ, A.bc_kind, A.bc_gamma, A.inv_h0, rv, e);
      if (KIND == 1) {
        // L^T Wb_k = -H (forward rows on yhat) + face terms, y = H yhat = P~ Wb_k at the node
        const T H = norm_weight_t<T, O>(i, d.nq) * A.h[0] * norm_weight_t<T, O>(j, d.nr) * A.h[1] *
                    norm_weight_t<T, O>(k, d.ns) * A.h[2];
        T vb[3], sb[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) vb[c] = -H * rv[c];
#pragma unroll
        for (int c = 0; c < 6; ++c) sb[c] = -H * e[c];
        if (face) {
          T y[9];
#pragma unroll
          for (int f = 0; f < 9; ++f) y[f] = H * qc[f];
          adjoint_face_terms(pos, N, a, y, irhoJ, lamJ, muJ, A.bc_kind, A.bc_gamma, A.inv_h0, vb, sb);
        }
        const T m9[9] = {vb[0], vb[1], vb[2], sb[0], sb[1], sb[2], sb[3], sb[4], sb[5]};
        if (A.mode == kModeRhs) {
#pragma unroll
          for (int f = 0; f < 9; ++f) fldw(ub_out, f)[off] = m9[f];
        } else if (!A.yhat_next) {
#pragma unroll
          for (int f = 0; f < 9; ++f) {
            fldw(ub_out, f)[off] = dqi[f] + A.dt * m9[f];
            fldw(wbm, f)[off] = A.rk_a * pre[f];
          }
        } else {
          // and the prep of stage k - 1, pointwise at this node: Wb_{k-1} = A_k Wb_k + B_{k-1} Ub_k,
          // yhat_{k-1} = H^-1 P~ Wb_{k-1} (1/H without a division)
          T w[9];
#pragma unroll
          for (int f = 0; f < 9; ++f) {
            const T ub = dqi[f] + A.dt * m9[f];
            fldw(ub_out, f)[off] = ub;
            w[f] = A.rk_a * pre[f] + A.rk_b_next * ub;
            fldw(wbm, f)[off] = w[f];
          }
          T y[9];
          apply_P(w, w + 3, irhoJ, lamJ, muJ, y);
          const T ih = norm_weight_inv_t<T, O>(i, d.nq) * A.inv_h[0] * norm_weight_inv_t<T, O>(j, d.nr) * A.inv_h[1] *
                       norm_weight_inv_t<T, O>(k, d.ns) * A.inv_h[2];
          T* yn = A.yhat_next + boff;
#pragma unroll
          for (int f = 0; f < 9; ++f) fldw(yn, f)[off] = y[f] * ih;
        }
      } else {
        // dt Wb_k . d(P~ M U_k)/d(rho, lambda, mu) at the node
        T y[9];
        if (face) {
          const T H = norm_weight_t<T, O>(i, d.nq) * A.h[0] * norm_weight_t<T, O>(j, d.nr) * A.h[1] *
                      norm_weight_t<T, O>(k, d.ns) * A.h[2];
#pragma unroll
          for (int f = 0; f < 9; ++f) y[f] = H * fld(yhm, f)[off];
        }
        double g[3];
        gradient_terms(rv, e, qc, pre, y, pos, N, a, irhoJ, lamJ, muJ, rj[0], rj[1], A.bc_kind, A.bc_gamma,
                       A.inv_h0, (double)A.dt, g);
        // one writer per node and launch: a reduction that needs no read-back
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(A.grad + c * fs + off, g[c]);
      }
    }
#pragma unroll
    for (int m = 0; m < NV - 1; ++m)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vq[m][c] = vq[m + 1][c];
        fq[m][c] = fq[m + 1][c];
      }
  }
}

// Self-test of the bounded wait used by the tiled kernel: one thread initialises an mbarrier
// that expects one arrival, nothing arrives, and the wait gives up after `polls` polls and
// records SBP_STATUS_TIMEOUT in the status word, exactly as the stage kernel does when a tile
// copy never lands.  The barrier lives in shared memory; nothing is left in flight.
__global__ void wait_selftest_kernel(unsigned polls, unsigned* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0, polls)) atomicOr(status, 8u);
}

cudaError_t launch_wait_selftest(unsigned polls, unsigned* status, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(polls, status);
  return cudaGetLastError();
}

// Planes a chunk spends filling its s queues before the first output plane.
template <int O>
constexpr int NVQ() { return OpCoef<O>::r + OpCoef<O>::q; }

template <typename T, int O, int KIND, int MAP = 0>
cudaError_t launch_tiled_order(const StageArgs<T>& A, const TmaSet& tm, cudaStream_t st) {
  const int ni = A.d.nq, nj = A.d.nr, nk = A.d.ns - A.slab.ghost_lo - A.slab.ghost_hi;  // computed planes
  // s chunks: at most 96 planes; when that leaves SM slots idle (few tiles), more chunks
  // (at least 16 planes each), the count that minimises waves x (chunk + queue warm-up)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;  // GB300
  const long long tiles = (long long)((ni + TX - 1) / TX) * ((nj + TY - 1) / TY) * A.nb;
  const long long slots = (long long)sms * tiled_min_blocks<T>();
  int nchunks = (nk + 95) / 96;
  if (tiles * nchunks < slots) {
    const int base = nchunks;
    long long best = -1;
    for (int nc = base; nc <= base + 8; ++nc) {
      const int ch = (nk + nc - 1) / nc;
      if (nc > base && ch < 16) break;
      const long long waves = (tiles * ((nk + ch - 1) / ch) + slots - 1) / slots;
      const long long cost = waves * (ch + NVQ<O>());
      if (best < 0 || cost < best) {
        best = cost;
        nchunks = nc;
      }
    }
  }
  const int chunk = (nk + nchunks - 1) / nchunks;
  dim3 grid((ni + TX - 1) / TX, (nj + TY - 1) / TY, ((nk + chunk - 1) / chunk) * A.nb);
  if (grid.z > 65535 || grid.y > 65535) return cudaErrorInvalidConfiguration;
  dim3 block(TX, TY);
  const size_t smem = sizeof(TiledShared<T, MAP>);
  cudaError_t e = cudaFuncSetAttribute(stage_tiled_kernel<T, O, KIND, MAP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  stage_tiled_kernel<T, O, KIND, MAP><<<grid, block, smem, st>>>(A, chunk, tm);
  return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t launch_kind(const StageArgs<T>& A, int order, const TmaSet& tm, cudaStream_t st) {
  if (!A.sclose) return cudaErrorInvalidValue;
  // the stage and the adjoint passes on a topography map: 4 metric fields (upwind orders 2, 4, 6);
  // the forward stage also takes the RK register with the plane (MAP 2)
  constexpr int kTopo = KIND == 0 ? 2 : 1;
  if (A.map == 1) {
    switch (order) {
      case 2: return launch_tiled_order<T, 2, KIND, kTopo>(A, tm, st);
      case 4: return launch_tiled_order<T, 4, KIND, kTopo>(A, tm, st);
      case 6: return launch_tiled_order<T, 6, KIND, kTopo>(A, tm, st);
      default: break;
    }
  }
  switch (order) {
    case 2: return launch_tiled_order<T, 2, KIND>(A, tm, st);
    case 4: return launch_tiled_order<T, 4, KIND>(A, tm, st);
    case 6: return launch_tiled_order<T, 6, KIND>(A, tm, st);
    default: break;
  }
  // the odd orders of Table 1 and the traditional operators of Table 2: forward stage only
  if constexpr (KIND == 0) {
    switch (order) {
      case 3: return launch_tiled_order<T, 3, 0>(A, tm, st);
      case 5: return launch_tiled_order<T, 5, 0>(A, tm, st);
      case 7: return launch_tiled_order<T, 7, 0>(A, tm, st);
      case kTraditional + 2: return launch_tiled_order<T, kTraditional + 2, 0>(A, tm, st);
      case kTraditional + 4: return launch_tiled_order<T, kTraditional + 4, 0>(A, tm, st);
      case kTraditional + 6: return launch_tiled_order<T, kTraditional + 6, 0>(A, tm, st);
      default: break;
    }
  }
  return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_stage_tiled(const StageArgs<T>& A, int order, const TmaSet& tm, cudaStream_t st) {
  return launch_kind<T, 0>(A, order, tm, st);
}

template <typename T>
cudaError_t launch_adjoint_tiled(const StageArgs<T>& A, int order, int pass, const TmaSet& tm, cudaStream_t st) {
  if (pass == 1) {
    if (!A.ubar_out || (A.mode != kModeRhs && !A.wbar)) return cudaErrorInvalidValue;
    return launch_kind<T, 1>(A, order, tm, st);
  }
  if (pass == 2) {
    if (!A.wbar || !A.yhat || !A.rlmj || !A.grad) return cudaErrorInvalidValue;
    return launch_kind<T, 2>(A, order, tm, st);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_stage_tiled<float>(const StageArgs<float>&, int, const TmaSet&, cudaStream_t);
template cudaError_t launch_stage_tiled<double>(const StageArgs<double>&, int, const TmaSet&, cudaStream_t);
template cudaError_t launch_adjoint_tiled<float>(const StageArgs<float>&, int, int, const TmaSet&, cudaStream_t);
template cudaError_t launch_adjoint_tiled<double>(const StageArgs<double>&, int, int, const TmaSet&, cudaStream_t);

}  // namespace sbp
