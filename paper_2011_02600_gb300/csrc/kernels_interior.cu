// Tiled interior stage kernel: nodes whose three axes all use interior stencil
// rows, i.e. the box [b, N-1-b] on every axis (b closure rows per face).
//
// Layout of the work: a block owns a TX x TY tile of the (q, r) plane and
// marches along s through a chunk of planes.
//   * q and r derivatives: each plane's flux F_q = sigma a_q, F_r = sigma a_r and
//     the velocity v are staged in shared memory with a halo of q (=max reach)
//     nodes; D-_q F_q, D+_q v, D-_r F_r, D+_r v read the tiles.
//   * s derivatives: every thread keeps register queues of its own column,
//     F_s = sigma a_s on planes k-q..k+r and v on planes k-r..k+q, so D-_s and
//     D+_s need no shared memory; the lead values v(k+q), sigma(k+r), a_s(k+r)
//     are the only loads that run ahead of the plane.
// The stage update (2N-storage Runge-Kutta) is fused in the epilogue.
#include "common.cuh"
#include "launch.h"

namespace sbp {

constexpr int TX = 32;
constexpr int TY = 8;

template <typename T, int O>
struct InteriorSmem {
  static constexpr int H = OpCoef<O>::q;  // max(r, q): the halo width
  T fq[3][TY][TX + 2 * H];
  T fr[3][TY + 2 * H][TX];
  T v[3][TY + 2 * H][TX + 2 * H];
};

// Two resident blocks per SM in FP32 (<= 128 registers a thread); FP64 needs the full register file.
template <typename T>
constexpr int interior_min_blocks() { return sizeof(T) == 4 ? 2 : 1; }

template <typename T, int O>
__global__ void __launch_bounds__(TX* TY, interior_min_blocks<T>())
    stage_interior_kernel(StageArgs<T> A, Box box, int chunk) {
  using C = OpCoef<O>;
  constexpr int R = C::r;    // D+ reaches -R..+Q, D- reaches -Q..+R
  constexpr int Q = C::q;
  constexpr int H = Q;
  constexpr int NV = R + Q + 1;  // queue length
  __shared__ InteriorSmem<T, O> sm;

  const Dims d = A.d;
  const long long fs = d.fs;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int i0 = box.i0 + blockIdx.x * TX;
  const int j0 = box.j0 + blockIdx.y * TY;
  const int i = i0 + tx, j = j0 + ty;
  const int kb = box.k0 + blockIdx.z * chunk;
  const int ke = min(box.k1, kb + chunk);
  const bool in_grid = i < d.nq && j < d.nr;
  const bool active = i < box.i1 && j < box.j1;
  const T ihq = A.inv_h[0], ihr = A.inv_h[1], ihs = A.inv_h[2];

  const T* __restrict__ q = A.q;
  const T* __restrict__ met = A.met;
  const int col = j * d.ldq + i;  // in-plane offset of this thread's column

  auto ld = [&](const T* p, long long off) -> T { return in_grid ? __ldg(p + off) : T(0); };

  // register queues of the thread's column
  T vq[NV][3];   // v at planes k-R .. k+Q
  T fq[NV][3];   // F_s at planes k-Q .. k+R
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

  for (int k = kb; k < ke; ++k) {
    const long long pk = (long long)k * d.plane;
    // lead values for the s queues
    {
      const long long offv = pk + (long long)Q * d.plane + col;
#pragma unroll
      for (int c = 0; c < 3; ++c) vq[NV - 1][c] = ld(q, c * fs + offv);
      const long long offf = pk + (long long)R * d.plane + col;
      T s[6], a[3];
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c] = ld(q, (3 + c) * fs + offf);
#pragma unroll
      for (int c = 0; c < 3; ++c) a[c] = ld(met, (6 + c) * fs + offf);
      flux(a, s, fq[NV - 1]);
    }
    // this plane's centre values
    const long long off = pk + col;
    T sc[6], aq[3], ar[3], as[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) sc[c] = ld(q, (3 + c) * fs + off);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      aq[c] = ld(met, c * fs + off);
      ar[c] = ld(met, (3 + c) * fs + off);
      as[c] = ld(met, (6 + c) * fs + off);
    }
    // stage the tiles: centre
    {
      T F[3];
      flux(aq, sc, F);
#pragma unroll
      for (int c = 0; c < 3; ++c) sm.fq[c][ty][H + tx] = F[c];
      flux(ar, sc, F);
#pragma unroll
      for (int c = 0; c < 3; ++c) sm.fr[c][H + ty][tx] = F[c];
#pragma unroll
      for (int c = 0; c < 3; ++c) sm.v[c][H + ty][H + tx] = vq[R][c];
    }
    // halo along r: rows -H..-1 and TY..TY+H-1, all TX columns (2*H*TX nodes)
    for (int t = tid; t < 2 * H * TX; t += TX * TY) {
      const int hr = t / TX, hc = t % TX;
      const int row = hr < H ? hr - H : TY + (hr - H);   // relative row
      const int gi = i0 + hc, gj = j0 + row;
      const bool ok = gi < d.nq && gj >= 0 && gj < d.nr;
      const long long o = pk + (long long)gj * d.ldq + gi;
      const bool needF = row >= -Q && row <= TY - 1 + R;
      const bool needV = row >= -R && row <= TY - 1 + Q;
      if (needF) {
        T s[6], a[3], F[3];
#pragma unroll
        for (int c = 0; c < 6; ++c) s[c] = ok ? __ldg(q + (3 + c) * fs + o) : T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) a[c] = ok ? __ldg(met + (3 + c) * fs + o) : T(0);
        flux(a, s, F);
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.fr[c][H + row][hc] = F[c];
      }
      if (needV) {
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.v[c][H + row][H + hc] = ok ? __ldg(q + c * fs + o) : T(0);
      }
    }
    // halo along q: columns -H..-1 and TX..TX+H-1, all TY rows (2*H*TY nodes)
    for (int t = tid; t < 2 * H * TY; t += TX * TY) {
      const int hc = t % (2 * H), hr = t / (2 * H);
      const int cc = hc < H ? hc - H : TX + (hc - H);    // relative column
      const int gi = i0 + cc, gj = j0 + hr;
      const bool ok = gi >= 0 && gi < d.nq && gj < d.nr;
      const long long o = pk + (long long)gj * d.ldq + gi;
      const bool needF = cc >= -Q && cc <= TX - 1 + R;
      const bool needV = cc >= -R && cc <= TX - 1 + Q;
      if (needF) {
        T s[6], a[3], F[3];
#pragma unroll
        for (int c = 0; c < 6; ++c) s[c] = ok ? __ldg(q + (3 + c) * fs + o) : T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) a[c] = ok ? __ldg(met + c * fs + o) : T(0);
        flux(a, s, F);
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.fq[c][hr][H + cc] = F[c];
      }
      if (needV) {
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.v[c][H + hr][H + cc] = ok ? __ldg(q + c * fs + o) : T(0);
      }
    }
    // epilogue inputs, issued before the barrier so their latency overlaps it
    T mt[3], dqi[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) mt[c] = ld(A.mat, c * fs + off);
    if (A.mode == kModeStage) {
#pragma unroll
      for (int c = 0; c < 9; ++c) dqi[c] = ld(A.dq, c * fs + off);
    }
    __syncthreads();

    T rv[3] = {T(0), T(0), T(0)};
    T e[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T dv[3];
    // q
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T sf = T(0), sv = T(0);
#pragma unroll
      for (int jj = -Q; jj <= R; ++jj) sf += T(-C::alpha(-jj)) * sm.fq[c][ty][H + tx + jj];
#pragma unroll
      for (int jj = -R; jj <= Q; ++jj) sv += T(C::alpha(jj)) * sm.v[c][H + ty][H + tx + jj];
      rv[c] += ihq * sf;
      dv[c] = ihq * sv;
    }
    add_strain(aq, dv, e);
    // r
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T sf = T(0), sv = T(0);
#pragma unroll
      for (int jj = -Q; jj <= R; ++jj) sf += T(-C::alpha(-jj)) * sm.fr[c][H + ty + jj][tx];
#pragma unroll
      for (int jj = -R; jj <= Q; ++jj) sv += T(C::alpha(jj)) * sm.v[c][H + ty + jj][H + tx];
      rv[c] += ihr * sf;
      dv[c] = ihr * sv;
    }
    add_strain(ar, dv, e);
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
    add_strain(as, dv, e);

    if (active) {
      T dd[9];
      apply_P(rv, e, mt[0], mt[1], mt[2], dd);
      const T qc[9] = {vq[R][0], vq[R][1], vq[R][2], sc[0], sc[1], sc[2], sc[3], sc[4], sc[5]};
      if (A.mode == kModeRhs) {
#pragma unroll
        for (int f = 0; f < 9; ++f) A.qout[f * fs + off] = dd[f];
      } else {
#pragma unroll
        for (int f = 0; f < 9; ++f) {
          T dn = A.dt * dd[f];
          if (A.mode == kModeStage) dn += A.rk_a * dqi[f];
          A.dq[f * fs + off] = dn;
          A.qout[f * fs + off] = qc[f] + A.rk_b * dn;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < NV - 1; ++m)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vq[m][c] = vq[m + 1][c];
        fq[m][c] = fq[m + 1][c];
      }
  }
}

template <typename T>
cudaError_t launch_stage_interior(const StageArgs<T>& A, int order, const Box& box, cudaStream_t st) {
  const int ni = box.i1 - box.i0, nj = box.j1 - box.j0, nk = box.k1 - box.k0;
  if (ni <= 0 || nj <= 0 || nk <= 0) return cudaErrorNotSupported;
  const int nchunks = (nk + 95) / 96;
  const int chunk = (nk + nchunks - 1) / nchunks;
  dim3 grid((ni + TX - 1) / TX, (nj + TY - 1) / TY, (nk + chunk - 1) / chunk);
  dim3 block(TX, TY);
  switch (order) {
    case 2: stage_interior_kernel<T, 2><<<grid, block, 0, st>>>(A, box, chunk); break;
    case 4: stage_interior_kernel<T, 4><<<grid, block, 0, st>>>(A, box, chunk); break;
    case 6: stage_interior_kernel<T, 6><<<grid, block, 0, st>>>(A, box, chunk); break;
    default: return cudaErrorNotSupported;
  }
  return cudaGetLastError();
}
template cudaError_t launch_stage_interior<float>(const StageArgs<float>&, int, const Box&, cudaStream_t);
template cudaError_t launch_stage_interior<double>(const StageArgs<double>&, int, const Box&, cudaStream_t);

}  // namespace sbp
