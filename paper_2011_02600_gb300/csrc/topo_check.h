// Per-node part of the topography-map check of sbp_set_material: how far the FP64 metrics jmet
// (J, then a[xi][eta] at field 1 + 3 xi + eta) at node t of the [s][r][q] enumeration are from
// those of a topography map x = L_x q, y = L_y r, z = z(q, r, s), where a_q = x_r x x_s =
// (L_y z_s, 0, 0) and a_r = x_s x x_q = (0, L_x z_s, 0) = (0, c a_q,x, 0) with c = L_x / L_y:
//   max( max(|a_q,y|, |a_q,z|, |a_r,x|, |a_r,z|) / |a_q,x|,  |a_r,y - c a_q,x| / |a_r,y| ),
// infinite where any of the six entries is not finite (fmax alone would drop a NaN) or the
// result is not.  Device code of the check kernel; without nvcc the same source compiles as
// host C++.
#pragma once

#include <math.h>

#include "common.cuh"

namespace sbp {

__host__ __device__ inline double topography_deviation(const double* jmet, const Dims& d, double c, long long t) {
  const int i = (int)(t % d.nq);
  const int j = (int)((t / d.nq) % d.nr);
  const int k = (int)(t / ((long long)d.nq * d.nr));
  const long long n0 = (long long)k * d.plane + (long long)j * d.ldq + i;
  const double aqx = jmet[1 * d.fs + n0], aqy = jmet[2 * d.fs + n0], aqz = jmet[3 * d.fs + n0];
  const double arx = jmet[4 * d.fs + n0], ary = jmet[5 * d.fs + n0], arz = jmet[6 * d.fs + n0];
  if (!(isfinite(aqx) && isfinite(aqy) && isfinite(aqz) && isfinite(arx) && isfinite(ary) && isfinite(arz)))
    return INFINITY;
  const double off = fmax(fmax(fabs(aqy), fabs(aqz)), fmax(fabs(arx), fabs(arz))) / fabs(aqx);
  const double ratio = fabs(ary - c * aqx) / fabs(ary);
  const double m = fmax(off, ratio);
  return m <= 1.0e300 ? m : INFINITY;  // NaN or infinite: not a topography map
}

}  // namespace sbp
