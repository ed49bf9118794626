// Tiled interior stage kernel: nodes whose three axes all use interior stencil
// rows (the box [b, N-1-b] on every axis; along q it starts at b rounded up to a
// multiple of 4 so that tile loads start on 16-byte boundaries).
//
// Work layout: a block owns a TX x TY tile of the (q, r) plane and marches along
// s through a chunk of planes.
//   * Plane data arrive by TMA, one plane ahead, into a two-stage shared-memory
//     ring: the 9 state fields with a halo of HX nodes on q and r, a_q with a q
//     halo, a_r with an r halo, a_s and the coefficients on the tile.  One
//     elected thread issues the copies; an mbarrier per stage counts the bytes.
//   * Each plane, the fluxes F_q = sigma a_q and F_r = sigma a_r are formed on the
//     tile and its halo into a double-buffered flux tile; one block barrier per
//     plane publishes them and frees the stage the next copy will overwrite.
//   * q and r derivatives read the flux and velocity tiles; s derivatives use
//     per-thread register queues of F_s = sigma a_s (planes k-q..k+r) and v
//     (planes k-r..k+q), fed by direct loads of the lead planes.
// The stage update (2N-storage Runge-Kutta) is fused in the epilogue.
#include "common.cuh"
#include "launch.h"
#include "tma.cuh"

namespace sbp {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int HX = 4;              // halo in the tile loads (>= q of every order)
constexpr int BXH = TX + 2 * HX;   // 40
constexpr int BYH = TY + 2 * HX;   // 16
constexpr unsigned kWaitLimit = 1u << 24;  // polls (with 64 ns sleeps) before giving up: about a second

template <typename T>
struct Stage {
  T state[9][BYH][BXH];
  T aq[3][TY][BXH];
  T ar[3][BYH][TX];
  T as[3][TY][TX];
  T mat[3][TY][TX];
};

template <typename T>
struct FluxTiles {
  T fq[3][TY][BXH];
  T fr[3][BYH][TX];
};

template <typename T>
struct InteriorShared {
  Stage<T> st[2];
  FluxTiles<T> f[2];
  unsigned long long bar[2];
};

template <typename T>
constexpr int interior_min_blocks() { return sizeof(T) == 4 ? 2 : 1; }

template <typename T>
__device__ __forceinline__ void issue_plane(InteriorShared<T>& S, int stage, const TmaSet& tm, int i0, int j0,
                                            int k, int member) {
  unsigned long long* bar = &S.bar[stage];
  mbar_expect_tx(bar, (unsigned)sizeof(Stage<T>));
  Stage<T>& st = S.st[stage];
  tma_load_4d(&st.state[0][0][0], &tm.state, i0 - HX, j0 - HX, k, 9 * member, bar);
  tma_load_4d(&st.aq[0][0][0], &tm.met_q, i0 - HX, j0, k, 0, bar);
  tma_load_4d(&st.ar[0][0][0], &tm.met_r, i0, j0 - HX, k, 3, bar);
  tma_load_4d(&st.as[0][0][0], &tm.met_s, i0, j0, k, 6, bar);
  tma_load_4d(&st.mat[0][0][0], &tm.mat, i0, j0, k, 0, bar);
}

template <typename T, int O>
__global__ void __launch_bounds__(TX* TY, interior_min_blocks<T>())
    stage_interior_kernel(StageArgs<T> A, Box box, int chunk, const __grid_constant__ TmaSet tm) {
  using C = OpCoef<O>;
  constexpr int R = C::r;    // D+ reaches -R..+Q, D- reaches -Q..+R
  constexpr int Q = C::q;
  constexpr int NV = R + Q + 1;
  static_assert(Q <= HX && R <= HX, "halo too small");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  InteriorShared<T>& S = *reinterpret_cast<InteriorShared<T>*>(smem_raw);

  const Dims d = A.d;
  const long long fs = d.fs;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int i0 = box.i0 + blockIdx.x * TX;
  const int j0 = box.j0 + blockIdx.y * TY;
  const int i = i0 + tx, j = j0 + ty;
  // blockIdx.z = chunk + nchunks * member (a batch of independent states)
  const int nchunks = gridDim.z / A.nb;
  const int member = blockIdx.z / nchunks;
  const int kb = box.k0 + (blockIdx.z % nchunks) * chunk;
  const int ke = min(box.k1, kb + chunk);
  const bool in_grid = i < d.nq && j < d.nr;
  const bool active = i < box.i1 && j < box.j1;
  const T ihq = A.inv_h[0], ihr = A.inv_h[1], ihs = A.inv_h[2];
  const long long boff = (long long)member * A.bstride;
  const T* __restrict__ q = A.q + boff;
  T* __restrict__ qout = A.qout + boff;
  T* __restrict__ dqm = A.dq + (A.mode == kModeRhs ? 0 : boff);
  const T* __restrict__ met = A.met;
  const int col = j * d.ldq + i;

  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) issue_plane(S, 0, tm, i0, j0, kb, member);

  auto ld = [&](const T* p, long long off) -> T { return in_grid ? __ldg(p + off) : T(0); };
  T vq[NV][3];  // v at planes k-R .. k+Q
  T fq[NV][3];  // F_s at planes k-Q .. k+R
#pragma unroll
  for (int m = 0; m < NV - 1; ++m) {
    const long long off = (long long)(kb - R + m) * d.plane + col;
#pragma unroll
    for (int c = 0; c < 3; ++c) vq[m][c] = ld(q, c * fs + off);
  }
#pragma unroll
  for (int m = 0; m < NV - 1; ++m) {
    const long long off = (long long)(kb - Q + m) * d.plane + col;
    T s[6], a[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c] = ld(q, (3 + c) * fs + off);
#pragma unroll
    for (int c = 0; c < 3; ++c) a[c] = ld(met, (6 + c) * fs + off);
    flux(a, s, fq[m]);
  }

  // lead values (v at k+Q, sigma and a_s at k+R) staged one plane ahead
  T lv[3], ls[6], la[3];
  auto load_lead = [&](int k) {
    const long long offv = (long long)(k + Q) * d.plane + col;
#pragma unroll
    for (int c = 0; c < 3; ++c) lv[c] = ld(q, c * fs + offv);
    const long long offf = (long long)(k + R) * d.plane + col;
#pragma unroll
    for (int c = 0; c < 6; ++c) ls[c] = ld(q, (3 + c) * fs + offf);
#pragma unroll
    for (int c = 0; c < 3; ++c) la[c] = ld(met, (6 + c) * fs + offf);
  };
  load_lead(kb);

  for (int it = 0, k = kb; k < ke; ++it, ++k) {
    const int sidx = it & 1;
    const unsigned phase = (it >> 1) & 1;
    const long long pk = (long long)k * d.plane;
    // push this plane's lead values (loaded during the previous plane), then fetch the next ones
#pragma unroll
    for (int c = 0; c < 3; ++c) vq[NV - 1][c] = lv[c];
    flux(la, ls, fq[NV - 1]);
    if (k + 1 < ke) load_lead(k + 1);
    const long long off = pk + col;
    T dqi[9];
    if (A.mode == kModeStage) {
#pragma unroll
      for (int c = 0; c < 9; ++c) dqi[c] = ld(dqm, c * fs + off);
    }

    if (!mbar_wait_bounded(&S.bar[sidx], phase, kWaitLimit)) {
      // The copy never completed (the only one in flight is the one waited for): record
      // it and leave; the host sees SBP_STATUS_TIMEOUT.
      if (tid == 0) atomicOr(A.status, 8u);
      return;
    }
    const Stage<T>& st = S.st[sidx];
    FluxTiles<T>& F = S.f[sidx];
    // fluxes on the tile and its halo: F_q at columns -Q..TX-1+R, F_r at rows -Q..TY-1+R
    for (int t = tid; t < TY * (Q + R + TX); t += TX * TY) {
      const int row = t / (Q + R + TX);
      const int cc = HX - Q + t % (Q + R + TX);
      const T a[3] = {st.aq[0][row][cc], st.aq[1][row][cc], st.aq[2][row][cc]};
      T s[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c] = st.state[3 + c][HX + row][cc];
      T Fv[3];
      flux(a, s, Fv);
#pragma unroll
      for (int c = 0; c < 3; ++c) F.fq[c][row][cc] = Fv[c];
    }
    for (int t = tid; t < TX * (Q + R + TY); t += TX * TY) {
      const int cl = t % TX;
      const int rr = HX - Q + t / TX;
      const T a[3] = {st.ar[0][rr][cl], st.ar[1][rr][cl], st.ar[2][rr][cl]};
      T s[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c] = st.state[3 + c][rr][HX + cl];
      T Fv[3];
      flux(a, s, Fv);
#pragma unroll
      for (int c = 0; c < 3; ++c) F.fr[c][rr][cl] = Fv[c];
    }
    __syncthreads();
    if (tid == 0 && k + 1 < ke) {
      fence_proxy_async_smem();
      issue_plane(S, sidx ^ 1, tm, i0, j0, k + 1, member);
    }

    T rv[3] = {T(0), T(0), T(0)};
    T e[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T dv[3];
    // q
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
    {
      const T a[3] = {st.aq[0][ty][HX + tx], st.aq[1][ty][HX + tx], st.aq[2][ty][HX + tx]};
      add_strain(a, dv, e);
    }
    // r
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
    {
      const T a[3] = {st.ar[0][HX + ty][tx], st.ar[1][HX + ty][tx], st.ar[2][HX + ty][tx]};
      add_strain(a, dv, e);
    }
    // s
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
    {
      const T a[3] = {st.as[0][ty][tx], st.as[1][ty][tx], st.as[2][ty][tx]};
      add_strain(a, dv, e);
    }

    if (active) {
      T dd[9];
      apply_P(rv, e, st.mat[0][ty][tx], st.mat[1][ty][tx], st.mat[2][ty][tx], dd);
      T qc[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) qc[c] = st.state[c][HX + ty][HX + tx];
      if (A.mode == kModeRhs) {
#pragma unroll
        for (int f = 0; f < 9; ++f) qout[f * fs + off] = dd[f];
      } else {
#pragma unroll
        for (int f = 0; f < 9; ++f) {
          T dn = A.dt * dd[f];
          if (A.mode == kModeStage) dn += A.rk_a * dqi[f];
          dqm[f * fs + off] = dn;
          qout[f * fs + off] = qc[f] + A.rk_b * dn;
        }
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

template <typename T, int O>
cudaError_t launch_interior_order(const StageArgs<T>& A, const Box& box, const TmaSet& tm, cudaStream_t st) {
  const int ni = box.i1 - box.i0, nj = box.j1 - box.j0, nk = box.k1 - box.k0;
  const int nchunks = (nk + 95) / 96;
  const int chunk = (nk + nchunks - 1) / nchunks;
  dim3 grid((ni + TX - 1) / TX, (nj + TY - 1) / TY, ((nk + chunk - 1) / chunk) * A.nb);
  if (grid.z > 65535 || grid.y > 65535) return cudaErrorInvalidConfiguration;
  dim3 block(TX, TY);
  const size_t smem = sizeof(InteriorShared<T>);
  cudaError_t e = cudaFuncSetAttribute(stage_interior_kernel<T, O>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  stage_interior_kernel<T, O><<<grid, block, smem, st>>>(A, box, chunk, tm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage_interior(const StageArgs<T>& A, int order, const Box& box, const TmaSet& tm,
                                  cudaStream_t st) {
  const int ni = box.i1 - box.i0, nj = box.j1 - box.j0, nk = box.k1 - box.k0;
  if (ni <= 0 || nj <= 0 || nk <= 0) return cudaErrorNotSupported;
  switch (order) {
    case 2: return launch_interior_order<T, 2>(A, box, tm, st);
    case 4: return launch_interior_order<T, 4>(A, box, tm, st);
    case 6: return launch_interior_order<T, 6>(A, box, tm, st);
    default: return cudaErrorNotSupported;
  }
}
template cudaError_t launch_stage_interior<float>(const StageArgs<float>&, int, const Box&, const TmaSet&,
                                                  cudaStream_t);
template cudaError_t launch_stage_interior<double>(const StageArgs<double>&, int, const Box&, const TmaSet&,
                                                   cudaStream_t);

}  // namespace sbp
