// The topography-map check's per-node body (topography_deviation of
// paper_2011_02600_gb300/csrc/topo_check.h) compiled as host C++: the largest deviation over a
// dense FP64 metric array (10 fields [s][r][q], no padding).  Built by tests/test_host_topography.py.
#include "topo_check.h"

extern "C" double host_topography_deviation(const double* jmet, int nq, int nr, int ns, double c) {
  const long long plane = (long long)nq * nr;
  const sbp::Dims d{nq, nr, ns, nq, (int)plane, plane * ns};
  double worst = 0.0;
  for (long long t = 0; t < plane * ns; ++t) worst = fmax(worst, sbp::topography_deviation(jmet, d, c, t));
  return worst;
}
